// Device helpers shared by the single-collection and the batched kernels (internal).
#pragma once

#include "skm_internal.cuh"

namespace skm {

// acc[q] += v * (two consecutive columns of the loaded row segment), one paired FP32
// fused multiply-add per two columns; each half rounds exactly like a scalar fmaf.
template <typename CT, int NV>
__device__ __forceinline__ void fma_row(float2 (&acc)[NV * 16 / (int)sizeof(CT) / 2], float v,
                                        const uint4 (&w)[NV]) {
    const float2 vv = make_float2(v, v);
#pragma unroll
    for (int u = 0; u < NV; ++u) {
        const uint32_t ww[4] = {w[u].x, w[u].y, w[u].z, w[u].w};
        if constexpr (sizeof(CT) == 4) {
            acc[u * 2 + 0] = __ffma2_rn(vv, make_float2(__uint_as_float(ww[0]), __uint_as_float(ww[1])), acc[u * 2 + 0]);
            acc[u * 2 + 1] = __ffma2_rn(vv, make_float2(__uint_as_float(ww[2]), __uint_as_float(ww[3])), acc[u * 2 + 1]);
        } else {
#pragma unroll
            for (int h = 0; h < 4; ++h)
                acc[u * 4 + h] = __ffma2_rn(vv, make_float2(bf16lo(ww[h]), bf16hi(ww[h])), acc[u * 4 + h]);
        }
    }
}

// Scoring of one document against one slice: acc (lane's J columns, as pairs) = sum over
// the nonzeros t in [beg, end), in CSR order, of x_t * C[t, lane columns] with one fused
// multiply-add per column. Cs points at the lane's first column of row 0; stage holds the
// warp's 32 staged (t, x) pairs. Rows of G nonzeros are loaded together.
template <typename CT, int NV>
__device__ __forceinline__ void slice_accumulate(int64_t beg, int64_t end, const int32_t *col, const float *val,
                                                 const CT *Cs, int64_t ldc, int2 *stage, int lane,
                                                 float2 (&acc)[NV * 16 / (int)sizeof(CT) / 2]) {
    constexpr int EPV = 16 / (int)sizeof(CT);
    constexpr int J = NV * EPV;
    constexpr int G = NV >= 4 ? 2 : 4;
#pragma unroll
    for (int q = 0; q < J / 2; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int64_t b = beg; b < end; b += 32) {
        const int n = (int)min((int64_t)32, end - b);
        __syncwarp();
        if (lane < n) stage[lane] = make_int2(__ldg(col + b + lane), __float_as_int(__ldg(val + b + lane)));
        __syncwarp();
        int q = 0;
        for (; q + G <= n; q += G) {
            uint4 w[G][NV];
            float v[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int2 tv = stage[q + g];
                v[g] = __int_as_float(tv.y);
                const CT *row = Cs + (int64_t)tv.x * ldc;
#pragma unroll
                for (int u = 0; u < NV; ++u) w[g][u] = ldg16(row + u * 32 * EPV);
            }
#pragma unroll
            for (int g = 0; g < G; ++g) fma_row<CT, NV>(acc, v[g], w[g]);
        }
        for (; q < n; ++q) {
            const int2 tv = stage[q];
            const CT *row = Cs + (int64_t)tv.x * ldc;
            uint4 w[NV];
#pragma unroll
            for (int u = 0; u < NV; ++u) w[u] = ldg16(row + u * 32 * EPV);
            fma_row<CT, NV>(acc, __int_as_float(tv.y), w);
        }
    }
}

// The slice's best TOPT (score, centroid id) of a warp's accumulators, written by lanes
// 0..TOPT-1 to part_s/part_j[o + lane]. Columns at or beyond ncols are ignored; col_ids maps
// a column to its centroid id (NULL: identity).
template <typename CT, int NV>
__device__ __forceinline__ void slice_topt_write(const float2 (&acc)[NV * 16 / (int)sizeof(CT) / 2], int64_t j0,
                                                 int lane, int32_t ncols, const int32_t *col_ids, float *part_s,
                                                 int32_t *part_j, int64_t o) {
    constexpr int EPV = 16 / (int)sizeof(CT);
    float ls[TOPT];
    int lj[TOPT];
#pragma unroll
    for (int q = 0; q < TOPT; ++q) { ls[q] = -INFINITY; lj[q] = INT32_MAX; }
#pragma unroll
    for (int u = 0; u < NV; ++u) {
#pragma unroll
        for (int e = 0; e < EPV; ++e) {
            const int64_t c = j0 + u * 32 * EPV + lane * EPV + e;
            if (c < ncols) {
                const int id = col_ids ? __ldg(col_ids + c) : (int)c;
                const int qq = (u * EPV + e) >> 1;
                topt_insert(ls, lj, (e & 1) ? acc[qq].y : acc[qq].x, id);
            }
        }
    }
    topt_warp_merge(ls, lj);
    if (lane < TOPT) {
        float s = ls[0];
        int j = lj[0];
#pragma unroll
        for (int q = 1; q < TOPT; ++q) if (lane == q) { s = ls[q]; j = lj[q]; }
        part_s[o + lane] = s;
        part_j[o + lane] = j;
    }
}

// Every column with score >= thr appended to cand[0..cap) (cnt counts all of them).
template <typename CT, int NV>
__device__ __forceinline__ void slice_collect(const float2 (&acc)[NV * 16 / (int)sizeof(CT) / 2], int64_t j0, int lane,
                                              int32_t ncols, const int32_t *col_ids, float thr, int32_t *cnt,
                                              int32_t *cand, int32_t cap) {
    constexpr int EPV = 16 / (int)sizeof(CT);
#pragma unroll
    for (int u = 0; u < NV; ++u) {
#pragma unroll
        for (int e = 0; e < EPV; ++e) {
            const int64_t c = j0 + u * 32 * EPV + lane * EPV + e;
            const int qq = (u * EPV + e) >> 1;
            const float sc = (e & 1) ? acc[qq].y : acc[qq].x;
            if (c < ncols && sc >= thr) {
                const int id = col_ids ? __ldg(col_ids + c) : (int)c;
                const int at = atomicAdd(cnt, 1);
                if (at < cap) cand[at] = id;
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// Error bound of the scoring pass for one document (all data are non-negative):
//   |s_hat - s| <= beta * s,  beta = u_c + gamma_n * (1 + u_c),
// u_c the unit roundoff of the centroid copy (2^-9 for BF16 round-to-nearest-even, 0 for
// the FP32 master itself) and gamma_n = n u / (1 - n u), u = 2^-24, n = nonzeros of the
// document (one rounding per fused multiply-add).
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double score_beta(int precision, int64_t nnz) {
    const double u = 5.9604644775390625e-08;  // 2^-24
    const double nu = (double)nnz * u;
    const double gam = nu / (1.0 - nu);
    const double uc = precision == 1 ? 1.953125e-03 : 0.0;  // 2^-9
    return uc + gam * (1.0 + uc);
}

// round(x * 2^F) for a finite x >= 0 from its bits (integer arithmetic only; ties round up)
__device__ __forceinline__ unsigned long long fixed_point(float x, int F) {
    const uint32_t b = __float_as_uint(x);
    const int e = (int)(b >> 23);
    if (e == 0 && (b & 0x7fffffu) == 0) return 0ull;
    const unsigned long long mant = (unsigned long long)((b & 0x7fffffu) | (e ? 0x800000u : 0u));
    const int sh = (e ? e : 1) - 150 + F;      // x = mant * 2^((e ? e : 1) - 150)
    if (sh >= 0) return mant << sh;
    if (sh <= -25) return 0ull;
    return (mant + (1ull << (-sh - 1))) >> (-sh);
}

// acc (two 64-bit words, low first) += x (hi:lo); order-independent exact 128-bit sum
__device__ __forceinline__ void atomic_add_u128(unsigned long long *acc, unsigned long long lo,
                                                unsigned long long hi) {
    const unsigned long long old = atomicAdd(acc, lo);
    hi += (old + lo < old) ? 1ull : 0ull;
    if (hi) atomicAdd(acc + 1, hi);
}

}  // namespace skm
