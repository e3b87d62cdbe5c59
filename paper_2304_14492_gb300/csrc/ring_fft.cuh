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
    static constexpr int TW_T1 = Q / 2 > 0 ? Q / 2 : 1;
    static constexpr int TW_FLOAT2 = TW_T1 + Q * L + (LOGL > 0 ? LOGL : 1) * L;

    __device__ static __forceinline__ void load_twiddles(float2* tab, const float2* __restrict__ tw) {
        float2* t1 = tab;
        float2* t2 = tab + TW_T1;
        float2* t3 = t2 + Q * L;
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
        const float2* t1 = tab;
        const float2* t2 = tab + TW_T1;
        const float2* t3 = t2 + Q * L;
#pragma unroll
        for (int h = Q / 2; h >= 1; h >>= 1) {
#pragma unroll
            for (int b = 0; b < Q; b += 2 * h) {
#pragma unroll
                for (int j = 0; j < h; ++j) {
                    const float2 x = v[b + j], y = v[b + j + h];
                    v[b + j] = cadd(x, y);
                    const float2 d = csub(x, y);
                    v[b + j + h] = (j == 0) ? d : cmul(d, t1[j * (Q / (2 * h))]);
                }
            }
        }
        const int tl = t & (L - 1);
#pragma unroll
        for (int r = 1; r < Q; ++r) v[r] = cmul(v[r], t2[brev_c<LOGQ>(r) * L + tl]);
#pragma unroll
        for (int lg = LOGL - 1; lg >= 0; --lg) {
            const int h = 1 << lg;
            const bool upper = (t & h) != 0;
            const float2 w = t3[lg * L + tl];
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                float2 p;
                p.x = __shfl_xor_sync(0xffffffffu, v[r].x, h);
                p.y = __shfl_xor_sync(0xffffffffu, v[r].y, h);
                v[r] = upper ? cmul(csub(p, v[r]), w) : cadd(v[r], p);
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
        const float2* t1 = tab;
        const float2* t2 = tab + TW_T1;
        const float2* t3 = t2 + Q * L;
        const int tl = t & (L - 1);
#pragma unroll
        for (int lg = 0; lg < LOGL; ++lg) {
            const int h = 1 << lg;
            const bool upper = (t & h) != 0;
            const float2 w = cconj(t3[lg * L + tl]);
#pragma unroll
            for (int r = 0; r < Q; ++r) {
                float2 p;
                p.x = __shfl_xor_sync(0xffffffffu, v[r].x, h);
                p.y = __shfl_xor_sync(0xffffffffu, v[r].y, h);
                v[r] = upper ? csub(p, cmul(w, v[r])) : cadd(v[r], cmul(w, p));
            }
        }
#pragma unroll
        for (int a = 1; a < Q; ++a) v[a] = cmul(v[a], cconj(t2[a * L + tl]));
#pragma unroll
        for (int h = Q / 2; h >= 1; h >>= 1) {
#pragma unroll
            for (int b = 0; b < Q; b += 2 * h) {
#pragma unroll
                for (int j = 0; j < h; ++j) {
                    const float2 x = v[b + j], y = v[b + j + h];
                    v[b + j] = cadd(x, y);
                    const float2 d = csub(x, y);
                    v[b + j + h] = (j == 0) ? d : cmul(d, cconj(t1[j * (Q / (2 * h))]));
                }
            }
        }
    }

    // Position (in float2 units, unpadded) of register r of lane t after forward().
    __device__ static __forceinline__ int out_index(int r, int t) {
        return brev_c<LOGQ>(r) + Q * brev_lane(t & (L - 1));
    }
};

}  // namespace zm
