// The angular sums of Eq. 1 as a matrix product: F_m(rho_i) = sum_k f_ik W_mk
// with W_mk = e^{-j m theta_k}, theta_k = 2 pi k / N_theta.  The tensor-core
// kernels (ring_dft.cu, polar_dft.cu) read W in tiles of KD angles, one tile
// per stage of their K loop, as the B operand of tcgen05.mma (kind::f16):
//
//   tile c, half h (bf16 hi / lo), row j, angle k (0 <= k < KD):
//     j <  ncols:  cos(m theta_{KD c + k}),  m = j
//     j >= ncols: -sin(m theta_{KD c + k}),  m = j - ncols
//   (zero where m > n_max), with ncols = 8 * ceil((n_max + 1) / 8), so the
//   MMA's N = 2 ncols puts Re F_m in accumulator column m and Im F_m in
//   column ncols + m.
//
// Each tile is stored in the canonical K-major, no-swizzle layout: 8-row
// groups of KD / 8 core matrices (8 rows x 16 bytes), core matrices adjacent
// in K 128 bytes apart, 8-row groups KD * 16 bytes apart; tile c half h
// starts at (2 c + h) * 2 ncols * KD * 2 bytes.  The angle index m k is
// reduced mod N_theta in integers and the sine and cosine are evaluated in
// FP64 before the split, so W_hi + W_lo is W to the split's 2^-16.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace zm {

template <int KD>
__host__ __device__ inline uint32_t dft_tile_off(int row, int k) {
    return (uint32_t)((row >> 3) * (KD * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

inline int dft_ncols(int n_max) { return 8 * ((n_max + 1 + 7) / 8); }

template <int KD>
inline size_t dft_table_bytes(int n_theta, int n_max) {
    return (size_t)(n_theta / KD) * 2 * (size_t)(2 * dft_ncols(n_max)) * KD * 2;
}

// One block per tile.
template <int KD>
__global__ void k_build_dft_tiles(int n_theta, int n_max, int ncols, uint8_t* __restrict__ out) {
    const int c = blockIdx.x;
    const int ncol2 = 2 * ncols;
    const size_t bt = (size_t)ncol2 * KD * 2;
    for (int e = threadIdx.x; e < ncol2 * KD; e += blockDim.x) {
        const int j = e / KD, k = e - j * KD;
        const int m = j < ncols ? j : j - ncols;
        double w = 0.0;
        if (m <= n_max) {
            const long long idx = ((long long)m * (KD * c + k)) % n_theta;
            double sn, cn;
            sincospi(2.0 * (double)idx / n_theta, &sn, &cn);
            w = j < ncols ? cn : -sn;
        }
        const __nv_bfloat16 hi = __double2bfloat16(w);
        const __nv_bfloat16 lo = __double2bfloat16(w - (double)__bfloat162float(hi));
        const uint32_t o = dft_tile_off<KD>(j, k);
        *reinterpret_cast<__nv_bfloat16*>(out + (size_t)c * 2 * bt + o) = hi;
        *reinterpret_cast<__nv_bfloat16*>(out + (size_t)c * 2 * bt + bt + o) = lo;
    }
}

}  // namespace zm
