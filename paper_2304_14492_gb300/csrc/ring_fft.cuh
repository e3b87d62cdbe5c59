// Warp-level complex FFT used for the per-ring angular transform.
//
// The angular factor e^{-j m theta} of Eq. 1 on theta_k = 2 pi k / N is a DFT
// over k; only m = 0..n_max is needed and the samples are real, so a ring of N
// real samples is packed into M = N/2 complex points z_j = x_{2j} + i x_{2j+1}
// and transformed with one M-point FFT per warp (the symmetry of e^{-j m theta}
// that the paper's Sec. 2 names as one of the two speed-ups).
//
// Decomposition M = Q * L (L = min(M, 32) lanes, Q points per lane): lane t
// holds z[t + L s], s = 0..Q-1.  (1) a Q-point DIF FFT over s in registers,
// (2) twiddles W_M^{t k1}, (3) an L-point DIF FFT over t across lanes with
// shuffles.  Lane t, register r then holds X[brev_Q(r) + Q brev_L(t)].
#pragma once

#include <cuda_runtime.h>

namespace zm {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// e^{-2 pi i x / 32} for x in [0, 32), from cos(pi k / 16), k = 0..8 and the
// quadrant symmetries.  Only for x known at compile time (after unrolling),
// where the table folds into immediates.
__device__ __forceinline__ float2 w32c(int x) {
    constexpr float C[9] = {1.0f, 0.98078528040323043f, 0.92387953251128674f, 0.83146961230254524f,
                            0.70710678118654752f, 0.55557023301960218f, 0.38268343236508977f,
                            0.19509032201612826f, 0.0f};
    float c, s;
    if (x <= 8) {
        c = C[x];
        s = C[8 - x];
    } else if (x <= 16) {
        c = -C[16 - x];
        s = C[x - 8];
    } else if (x <= 24) {
        c = -C[x - 16];
        s = -C[24 - x];
    } else {
        c = C[32 - x];
        s = -C[x - 24];
    }
    return make_float2(c, -s);
}

// d * W_32^x (d * conj(W_32^x) for INV) with x known at compile time; the
// quarter turns cost no multiplication.
template <bool INV>
__device__ __forceinline__ float2 mul_w32(float2 d, int x) {
    x &= 31;
    if (x == 0) return d;
    if (x == 16) return make_float2(-d.x, -d.y);
    if (x == 8) return INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);    // * (+i) : * (-i)
    if (x == 24) return INV ? make_float2(d.y, -d.x) : make_float2(-d.y, d.x);   // * (-i) : * (+i)
    const float2 w = w32c(x);
    return cmul(d, INV ? cconj(w) : w);
}

template <int BITS>
__host__ __device__ constexpr int brev_c(int x) {
    int r = 0;
    for (int b = 0; b < BITS; ++b) r |= ((x >> b) & 1) << (BITS - 1 - b);
    return r;
}

template <int LOGN>
struct RingFFT {
    static constexpr int N = 1 << LOGN;              // real ring length
    static constexpr int LOGM = LOGN - 1;
    static constexpr int M = 1 << LOGM;              // complex points
    static constexpr int LOGL = LOGM < 5 ? LOGM : 5;
    static constexpr int L = 1 << LOGL;              // lanes carrying data
    static constexpr int LOGQ = LOGM - LOGL;
    static constexpr int Q = 1 << LOGQ;              // points per lane
    // Row of M float2 with one float2 of padding per 16 (bank spread for the
    // bit-reversed stores): N + N/8 floats, rounded up to a multiple of 4 so
    // that every row starts 16-byte aligned.
    static constexpr int ROW_FLOATS = ((N + N / 8 + 3) / 4) * 4;
    static_assert(ROW_FLOATS % 4 == 0, "ring rows must stay 16-byte aligned");
    static_assert(2 * (M + (M - 1) / 16) <= ROW_FLOATS, "padded spectrum must fit the row");

    // Twiddles used by one warp FFT, staged once per CTA in shared memory:
    //   t1[x]         = W_Q^x,               x < Q/2   (in-register stages)
    //   t2[k1 * L + t] = W_M^{t k1},          k1 < Q    (between the stages)
    //   t3[e * L + t]  = W_{2h}^{t mod h},    h = 2^e   (cross-lane stages)
    // with W_n = e^{-2 pi i / n}; the inverse uses their conjugates.
    //   t32[x]         = W_32^x,             x < 32    (transposed form only)
    static constexpr int TW_T1 = Q / 2 > 0 ? Q / 2 : 1;
    static constexpr int TW_T3 = (LOGL > 0 ? LOGL : 1) * L;
    static constexpr int TW_FLOAT2 = TW_T1 + Q * L + TW_T3 + 32;

    // Transposed form (Q >= 4, i.e. N >= 256): the 32-point DFTs across lanes
    // are done by G = 32/Q lanes each, so only log2(G) shuffle stages remain;
    // a per-warp shared buffer of TBUF float2 (rows of 33) carries the transpose.
    static constexpr bool TRANSPOSED = LOGQ >= 2;
    static constexpr int LOGG = TRANSPOSED ? 5 - LOGQ : 0;
    static constexpr int G = 1 << LOGG;
    static constexpr int TSTRIDE = 33;
    static constexpr int TBUF = TRANSPOSED ? Q * TSTRIDE : 0;

    // In-register Q-point DFT (decimation in frequency): v[r] becomes the
    // transform at index brev_Q(r); INV uses e^{+2 pi i / Q}.  The twiddle of
    // butterfly j at span h is W_Q^{j Q / 2h} = W_32^{16 j / h}, an immediate.
    template <bool INV>
    __device__ static __forceinline__ void reg_dft(float2 (&v)[Q], const float2*) {
        static_assert(Q <= 32, "in-register DFTs up to 32 points");
#pragma unroll
        for (int h = Q / 2; h >= 1; h >>= 1) {
#pragma unroll
            for (int b = 0; b < Q; b += 2 * h) {
#pragma unroll
                for (int j = 0; j < h; ++j) {
                    const float2 x = v[b + j], y = v[b + j + h];
                    v[b + j] = cadd(x, y);
                    v[b + j + h] = mul_w32<INV>(csub(x, y), 16 * j / h);
                }
            }
        }
    }

    __device__ static __forceinline__ void load_twiddles(float2* tab, const float2* __restrict__ tw) {
        float2* t1 = tab;
        float2* t2 = tab + TW_T1;
        float2* t3 = t2 + Q * L;
        float2* t32 = t3 + TW_T3;
        for (int x = threadIdx.x; x < 32; x += blockDim.x) t32[x] = N >= 32 ? __ldg(&tw[x * (N >= 32 ? N / 32 : 1)]) : make_float2(1.f, 0.f);
        for (int x = threadIdx.x; x < Q / 2; x += blockDim.x) t1[x] = __ldg(&tw[x * (N / Q)]);
        for (int e = threadIdx.x; e < Q * L; e += blockDim.x) {
            const int k1 = e / L, t = e - k1 * L;
            t2[e] = __ldg(&tw[2 * t * k1]);
        }
        for (int e = threadIdx.x; e < LOGL * L; e += blockDim.x) {
            const int lg = e / L, t = e - lg * L;
            const int h = 1 << lg;
            t3[e] = __ldg(&tw[(t & (h - 1)) * (N / (2 * h))]);
        }
    }

    __device__ static __forceinline__ int pad(int j) { return j + (j >> 4); }
    __device__ static __forceinline__ int brev_lane(int t) {
        return LOGL == 0 ? 0 : (int)(__brev((unsigned)t) >> (32 - LOGL));
    }

    // Forward DFT X_k = sum_j z_j e^{-2 pi i j k / M}; `tab` from
    // load_twiddles().  All 32 lanes must call; lanes >= L carry dummy data.
    __device__ static __forceinline__ void forward(float2 (&v)[Q], int t, const float2* tab) {
        const float2* t2 = tab + TW_T1;
        const float2* t3 = t2 + Q * L;
        reg_dft<false>(v, tab);
        const int tl = t & (L - 1);
#pragma unroll
        for (int r = 1; r < Q; ++r) v[r] = cmul(v[r], t2[brev_c<LOGQ>(r) * L + tl]);
#pragma unroll
        for (int lg = LOGL - 1; lg >= 0; --lg) {
            const int h = 1 << lg;
            const bool upper = (t & h) != 0;
            const float2 w = t3[lg * L + tl];      // W_2h^{t mod h}; 1 at h = 1
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                float2 p;
                p.x = __shfl_xor_sync(0xffffffffu, v[r].x, h);
                p.y = __shfl_xor_sync(0xffffffffu, v[r].y, h);
                if (h == 1) v[r] = upper ? csub(p, v[r]) : cadd(v[r], p);
                else v[r] = upper ? cmul(csub(p, v[r]), w) : cadd(v[r], p);
            }
        }
    }

    // Inverse DFT z_j = sum_m C_m e^{+2 pi i j m / M} in the transposed
    // structure: on entry lane l, register a holds C[a + Q brev_L(l)]; on exit
    // lane t, register r holds z[t + L brev_Q(r)] (natural order across lanes).
    // With m = a + Q c and j = t + L s:
    //   z[t + L s] = sum_a e^{2 pi i a s / Q} e^{2 pi i a t / M} sum_c C[a + Q c] e^{2 pi i c t / L},
    // i.e. an L-point DFT across lanes (decimation in time, bit-reversed input),
    // a twiddle, and a Q-point DFT in registers (decimation in frequency).
    __device__ static __forceinline__ void inverse_natural(float2 (&v)[Q], int t, const float2* tab) {
        const float2* t2 = tab + TW_T1;
        const float2* t3 = t2 + Q * L;
        const int tl = t & (L - 1);
#pragma unroll
        for (int lg = 0; lg < LOGL; ++lg) {
            const int h = 1 << lg;
            const bool upper = (t & h) != 0;
            const float2 w = cconj(t3[lg * L + tl]);     // 1 at h = 1
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                float2 p;
                p.x = __shfl_xor_sync(0xffffffffu, v[r].x, h);
                p.y = __shfl_xor_sync(0xffffffffu, v[r].y, h);
                if (h == 1) v[r] = upper ? csub(p, v[r]) : cadd(v[r], p);
                else v[r] = upper ? csub(p, cmul(w, v[r])) : cadd(v[r], cmul(w, p));
            }
        }
#pragma unroll
        for (int a = 1; a < Q; ++a) v[a] = cmul(v[a], cconj(t2[a * L + tl]));
        reg_dft<true>(v, tab);
    }

    __device__ static __forceinline__ int brev_g(int g) {
        return LOGG == 0 ? 0 : (int)(__brev((unsigned)g) >> (32 - LOGG));
    }

    // Transposed forward DFT.  In: lane t, register s = z[t + 32 s].  With
    // k = k1 + Q (a + Q b):  A) Q-point DFT over s, B) twiddle W_M^{t k1},
    // transpose so that lane (k1, g) (k1 = lane / G, g = lane mod G) holds
    // Y[k1][g + G u], u < Q;  C1) Q-point DFT over u, C2) twiddle W_32^{g a},
    // C3) G-point DFT across the group's lanes.  Out: see fwd_index().
    __device__ static __forceinline__ void forward_t(float2 (&v)[Q], int lane, const float2* tab, float2* buf) {
        const float2* t1 = tab;
        const float2* t2 = tab + TW_T1;
        const float2* t32 = t2 + Q * L + TW_T3;
        reg_dft<false>(v, t1);
#pragma unroll
        for (int r = 1; r < Q; ++r) v[r] = cmul(v[r], t2[brev_c<LOGQ>(r) * L + lane]);
        __syncwarp();
#pragma unroll
        for (int r = 0; r < Q; ++r) buf[brev_c<LOGQ>(r) * TSTRIDE + lane] = v[r];
        __syncwarp();
        const int k1 = lane >> LOGG, g = lane & (G - 1);
#pragma unroll
        for (int u = 0; u < Q; ++u) v[u] = buf[k1 * TSTRIDE + g + G * u];
        __syncwarp();
        reg_dft<false>(v, t1);
        if constexpr (G == 2) {
            // W_32^{g brev(r)}, g in {0, 1}: an immediate or 1
#pragma unroll
            for (int r = 1; r < Q; ++r) {
                const float2 m = mul_w32<false>(v[r], brev_c<LOGQ>(r));
                v[r] = g ? m : v[r];
            }
        } else if constexpr (G > 2) {
#pragma unroll
            for (int r = 1; r < Q; ++r) v[r] = cmul(v[r], t32[g * brev_c<LOGQ>(r)]);
        }
#pragma unroll
        for (int h = G / 2; h >= 1; h >>= 1) {
            const bool upper = (g & h) != 0;
            const float2 w = t32[(g & (h - 1)) * (16 / h)];     // 1 at h = 1
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                float2 p;
                p.x = __shfl_xor_sync(0xffffffffu, v[r].x, h);
                p.y = __shfl_xor_sync(0xffffffffu, v[r].y, h);
                if (h == 1) v[r] = upper ? csub(p, v[r]) : cadd(v[r], p);
                else v[r] = upper ? cmul(csub(p, v[r]), w) : cadd(v[r], p);
            }
        }
    }

    // Transposed inverse DFT z_j = sum_m C_m e^{+2 pi i j m / M}.  In: lane
    // (k1, g), register a = C[k1 + Q (a + Q brev_G(g))] (see inv_index()).
    // Out: lane t, register r = z[t + 32 brev_Q(r)] (natural across lanes).
    __device__ static __forceinline__ void inverse_t(float2 (&v)[Q], int lane, const float2* tab, float2* buf) {
        const float2* t1 = tab;
        const float2* t2 = tab + TW_T1;
        const float2* t32 = t2 + Q * L + TW_T3;
        const int k1 = lane >> LOGG, g = lane & (G - 1);
#pragma unroll
        for (int lg = 0; lg < LOGG; ++lg) {
            const int h = 1 << lg;
            const bool upper = (g & h) != 0;
            const float2 w = cconj(t32[(g & (h - 1)) * (16 / h)]);     // 1 at h = 1
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                float2 p;
                p.x = __shfl_xor_sync(0xffffffffu, v[r].x, h);
                p.y = __shfl_xor_sync(0xffffffffu, v[r].y, h);
                if (h == 1) v[r] = upper ? csub(p, v[r]) : cadd(v[r], p);
                else v[r] = upper ? csub(p, cmul(w, v[r])) : cadd(v[r], cmul(w, p));
            }
        }
        if constexpr (G == 2) {
#pragma unroll
            for (int a = 1; a < Q; ++a) {
                const float2 m = mul_w32<true>(v[a], a);
                v[a] = g ? m : v[a];
            }
        } else if constexpr (G > 2) {
#pragma unroll
            for (int a = 1; a < Q; ++a) v[a] = cmul(v[a], cconj(t32[g * a]));
        }
        reg_dft<true>(v, t1);
        __syncwarp();
#pragma unroll
        for (int r = 0; r < Q; ++r) buf[k1 * TSTRIDE + g + G * brev_c<LOGQ>(r)] = v[r];
        __syncwarp();
#pragma unroll
        for (int q = 0; q < Q; ++q) v[q] = buf[q * TSTRIDE + lane];
        __syncwarp();
#pragma unroll
        for (int q = 1; q < Q; ++q) v[q] = cmul(v[q], cconj(t2[q * L + lane]));
        reg_dft<true>(v, t1);
    }

    // Whichever form fits N: forward / inverse with their index maps.
    __device__ static __forceinline__ void fwd(float2 (&v)[Q], int lane, const float2* tab, float2* buf) {
        if constexpr (TRANSPOSED) forward_t(v, lane, tab, buf);
        else forward(v, lane, tab);
    }
    __device__ static __forceinline__ void inv(float2 (&v)[Q], int lane, const float2* tab, float2* buf) {
        if constexpr (TRANSPOSED) inverse_t(v, lane, tab, buf);
        else inverse_natural(v, lane, tab);
    }
    // index of the spectrum held in register r of `lane` after fwd()
    __device__ static __forceinline__ int fwd_index(int r, int lane) {
        if constexpr (TRANSPOSED) {
            const int k1 = lane >> LOGG, g = lane & (G - 1);
            return k1 + Q * (brev_c<LOGQ>(r) + Q * brev_g(g));
        } else {
            return out_index(r, lane);
        }
    }
    // index of the spectrum inv() expects in register a of `lane`
    __device__ static __forceinline__ int inv_index(int a, int lane) {
        if constexpr (TRANSPOSED) {
            const int k1 = lane >> LOGG, g = lane & (G - 1);
            return k1 + Q * (a + Q * brev_g(g));
        } else {
            return a + Q * brev_lane(lane & (L - 1));
        }
    }

    // Position (in float2 units, unpadded) of register r of lane t after forward().
    __device__ static __forceinline__ int out_index(int r, int t) {
        return brev_c<LOGQ>(r) + Q * brev_lane(t & (L - 1));
    }
};

}  // namespace zm
