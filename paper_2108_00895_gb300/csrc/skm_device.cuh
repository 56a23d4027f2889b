// Device helpers shared by the single-collection and the batched kernels (internal).
#pragma once

#include <type_traits>

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

// Sparse rows of one scoring slice. A term t whose centroid row is stored sparsely arrives
// in the column stream as ~t (negative); its nonzeros in this slice are ent[ptr[t * (n_slices
// + 1) + slice] .. ptr[... + 1]), ascending column: (offset within the slice << 16 | BF16
// bits) for BF16 matrices, {offset, FP32 bits} for FP32 ones; lists are padded to whole
// 16-byte vectors with entries for offset KS, a spare scratch column.
struct RareSlice {
    const uint32_t *ptr = nullptr;
    const void *ent = nullptr;
    int32_t n_slices = 0;
    int32_t slice = 0;
    int32_t cols = 0;                  // valid columns of this slice
    float *sacc = nullptr;             // the warp's scratch: one float per slice column + spare
    void *stg = nullptr;               // the warp's list staging: RARE_STAGE_BYTES
    unsigned long long skipped = 0;    // multiply-adds by exact zeros not executed (lane-uniform)
};

constexpr int RARE_STAGE_BYTES = 1024;
constexpr int RARE_SPARE = 4;          // scratch floats past the slice (16-byte multiple)

// Rows [q, qe) of the staged (t, x) pairs, all dense, accumulated in order; G rows are
// loaded together.
template <typename CT, int NV>
__device__ __forceinline__ void dense_rows(int q, int qe, const int2 *stage, const CT *Cs, int64_t ldc,
                                           float2 (&acc)[NV * 16 / (int)sizeof(CT) / 2]) {
    constexpr int EPV = 16 / (int)sizeof(CT);
    constexpr int G = NV >= 4 ? 2 : 4;
    for (; q + G <= qe; q += G) {
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
    for (; q < qe; ++q) {
        const int2 tv = stage[q];
        const CT *row = Cs + (int64_t)tv.x * ldc;
        uint4 w[NV];
#pragma unroll
        for (int u = 0; u < NV; ++u) w[u] = ldg16(row + u * 32 * EPV);
        fma_row<CT, NV>(acc, __int_as_float(tv.y), w);
    }
}

// Rows [q0, q1) of the staged pairs, all sparse, in order. The accumulators go through the
// warp's scratch: each nonzero (c, v) of a row updates column c with the same fused
// multiply-add the dense form would apply, and the zeros it skips would add exactly +0,
// so the result is bit-identical to accumulating the dense rows. Lane q holds the list
// bounds (e0, e1) and the value x of staged row q, loaded at staging time. The lanes copy
// their rows' lists into the staging buffer together (16-byte loads, one latency round
// for as many rows as fit), then the rows are applied one after another from shared
// memory; a list longer than the buffer is applied straight from global memory.
template <typename CT, int NV>
__device__ __forceinline__ void sparse_rows(int q0, int q1, RareSlice &rs, int lane, uint32_t e0_mine,
                                            uint32_t e1_mine, float x_mine,
                                            float2 (&acc)[NV * 16 / (int)sizeof(CT) / 2]) {
    constexpr int EPV = 16 / (int)sizeof(CT);
    using E = typename std::conditional<sizeof(CT) == 2, uint32_t, uint2>::type;
    constexpr uint32_t EV = 16 / sizeof(E);                       // entries per vector
    constexpr uint32_t CAP = RARE_STAGE_BYTES / sizeof(E);        // staged entries
    const E *ent = static_cast<const E *>(rs.ent);
    E *stg = static_cast<E *>(rs.stg);
    auto apply = [&](const E &w, float x) {
        if constexpr (sizeof(CT) == 2) {
            float *p = rs.sacc + (w >> 16);
            *p = fmaf(x, __uint_as_float(w << 16), *p);
        } else {
            float *p = rs.sacc + w.x;
            *p = fmaf(x, __uint_as_float(w.y), *p);
        }
    };
    float4 *mine = reinterpret_cast<float4 *>(rs.sacc + lane * EPV);
#pragma unroll
    for (int u = 0; u < NV; ++u)
#pragma unroll
        for (int h = 0; h < EPV / 4; ++h)
            mine[u * 8 * EPV + h] = make_float4(acc[u * EPV / 2 + 2 * h].x, acc[u * EPV / 2 + 2 * h].y,
                                                acc[u * EPV / 2 + 2 * h + 1].x, acc[u * EPV / 2 + 2 * h + 1].y);
    __syncwarp();
    const bool in_run = lane >= q0 && lane < q1;
    const uint32_t len_mine = in_run ? e1_mine - e0_mine : 0u;
    int q = q0;
    while (q < q1) {
        // rows [q, qc) whose lists fit in the buffer together
        uint32_t l = lane >= q ? len_mine : 0u;
        uint32_t incl = l;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += o;
        }
        const unsigned over = __ballot_sync(FULL, lane >= q && lane < q1 && incl > CAP);
        int qc = over ? __ffs(over) - 1 : q1;
        const bool direct = qc == q;          // row q alone overflows the buffer
        if (direct) qc = q + 1;
        if (!direct && lane >= q && lane < qc) {
            const uint32_t o = incl - l;
            const uint4 *src = reinterpret_cast<const uint4 *>(ent + e0_mine);
            uint4 *dst = reinterpret_cast<uint4 *>(stg + o);
#pragma unroll 4
            for (uint32_t v = 0; v < l / EV; ++v) dst[v] = __ldg(src + v);
        }
        __syncwarp();
        for (int r = q; r < qc; ++r) {
            const uint32_t len_r = __shfl_sync(FULL, l, r);
            const uint32_t off_r = __shfl_sync(FULL, incl - l, r);
            const uint32_t e0_r = __shfl_sync(FULL, e0_mine, r);
            const float x_r = __shfl_sync(FULL, x_mine, r);
            for (uint32_t e = lane; e < len_r; e += 32u) apply(direct ? __ldg(ent + e0_r + e) : stg[off_r + e], x_r);
            if ((uint32_t)rs.cols > len_r) rs.skipped += (unsigned long long)(rs.cols - len_r);
            __syncwarp();
        }
        q = qc;
    }
#pragma unroll
    for (int u = 0; u < NV; ++u)
#pragma unroll
        for (int h = 0; h < EPV / 4; ++h) {
            const float4 f = mine[u * 8 * EPV + h];
            acc[u * EPV / 2 + 2 * h] = make_float2(f.x, f.y);
            acc[u * EPV / 2 + 2 * h + 1] = make_float2(f.z, f.w);
        }
    __syncwarp();
}

// acc (lane's J columns, as pairs) += x_t * C[t, lane columns] for the nonzeros t in
// [beg, end), in CSR order, one fused multiply-add per column and nonzero. Cs points at the
// lane's first column of row 0; stage holds the warp's 32 staged (t, x) pairs. Rows of G
// nonzeros are loaded together.
template <typename CT, int NV>
__device__ __forceinline__ void slice_accumulate_add(int64_t beg, int64_t end, const int32_t *col, const float *val,
                                                     const CT *Cs, int64_t ldc, int2 *stage, int lane,
                                                     float2 (&acc)[NV * 16 / (int)sizeof(CT) / 2]) {
    constexpr int EPV = 16 / (int)sizeof(CT);
    constexpr int G = NV >= 4 ? 2 : 4;
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

// Scoring of one document against one slice: acc = sum over the nonzeros in [beg, end), in
// CSR order, of x_t * C[t, lane columns] (slice_accumulate_add from zero).
template <typename CT, int NV>
__device__ __forceinline__ void slice_accumulate(int64_t beg, int64_t end, const int32_t *col, const float *val,
                                                 const CT *Cs, int64_t ldc, int2 *stage, int lane,
                                                 float2 (&acc)[NV * 16 / (int)sizeof(CT) / 2]) {
    constexpr int J = NV * 16 / (int)sizeof(CT);
#pragma unroll
    for (int q = 0; q < J / 2; ++q) acc[q] = make_float2(0.f, 0.f);
    slice_accumulate_add<CT, NV>(beg, end, col, val, Cs, ldc, stage, lane, acc);
}

// slice_accumulate with sparse rows: negative column entries ~t mark rows stored by their
// nonzeros (see RareSlice); runs of dense and sparse rows alternate in CSR order, so every
// score is the one slice_accumulate computes from the dense matrix, bit for bit. With
// from_zero = false the chain continues from the given accumulators (head sums).
template <typename CT, int NV>
__device__ __forceinline__ void slice_accumulate_sparse(int64_t beg, int64_t end, const int32_t *col,
                                                        const float *val, const CT *Cs, int64_t ldc, int2 *stage,
                                                        int lane, float2 (&acc)[NV * 16 / (int)sizeof(CT) / 2],
                                                        RareSlice &rs, bool from_zero = true) {
    constexpr int EPV = 16 / (int)sizeof(CT);
    constexpr int J = NV * EPV;
    if (from_zero)
#pragma unroll
        for (int q = 0; q < J / 2; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int64_t b = beg; b < end; b += 32) {
        const int n = (int)min((int64_t)32, end - b);
        __syncwarp();
        int t_mine = 0;
        float x_mine = 0.f;
        uint32_t e0_mine = 0, e1_mine = 0;
        if (lane < n) {
            t_mine = __ldg(col + b + lane);
            x_mine = __ldg(val + b + lane);
            stage[lane] = make_int2(t_mine, __float_as_int(x_mine));
            if (t_mine < 0) {
                const uint32_t *pp = rs.ptr + (int64_t)(~t_mine) * (rs.n_slices + 1) + rs.slice;
                e0_mine = __ldg(pp);
                e1_mine = __ldg(pp + 1);
            }
        }
        __syncwarp();
        const unsigned rare = __ballot_sync(FULL, t_mine < 0);
        if (rare == 0u) {
            dense_rows<CT, NV>(0, n, stage, Cs, ldc, acc);
            continue;
        }
        const unsigned valid = n >= 32 ? FULL : ((1u << n) - 1u);
        int q = 0;
        while (q < n) {
            const unsigned r_from = rare & (FULL << q);
            const int qe = r_from ? __ffs(r_from) - 1 : n;
            dense_rows<CT, NV>(q, qe, stage, Cs, ldc, acc);
            if (qe >= n) break;
            const unsigned d_from = ~rare & valid & (FULL << qe);
            const int qr = d_from ? __ffs(d_from) - 1 : n;
            sparse_rows<CT, NV>(qe, qr, rs, lane, e0_mine, e1_mine, x_mine, acc);
            q = qr;
        }
    }
}

// The warp's best TOPT over the lanes' best-first lists, in TOPT rounds: the largest score,
// then the smallest id among the lanes that hold it; the winning lane drops its head. Scores
// are non-negative, so their bit patterns order like their values and one warp reduction
// finds the largest; an empty entry (-inf, INT32_MAX) and a score of +0 both count as 0, and
// the id decides, as in `better`. Every lane ends with the result in ls, lj, best first.
__device__ __forceinline__ void topt_warp_select(float (&ls)[TOPT], int (&lj)[TOPT]) {
    const int lane = threadIdx.x & 31;
    float rs[TOPT];
    int rj[TOPT];
#pragma unroll
    for (int q = 0; q < TOPT; ++q) {
        const uint32_t key = ls[0] > 0.f ? __float_as_uint(ls[0]) : 0u;
        const uint32_t kmax = __reduce_max_sync(FULL, key);
        const bool top = key == kmax;
        const unsigned holders = __ballot_sync(FULL, top);
        uint32_t jm = (uint32_t)lj[0];
        if (__popc(holders) > 1 && top) jm = __reduce_min_sync(holders, (uint32_t)lj[0]);
        const int win = __ffs(__ballot_sync(FULL, top && (uint32_t)lj[0] == jm)) - 1;
        rs[q] = __shfl_sync(FULL, ls[0], win);
        rj[q] = __shfl_sync(FULL, lj[0], win);
        if (lane == win) {
#pragma unroll
            for (int r = 0; r + 1 < TOPT; ++r) {
                ls[r] = ls[r + 1];
                lj[r] = lj[r + 1];
            }
            ls[TOPT - 1] = -INFINITY;
            lj[TOPT - 1] = INT32_MAX;
        }
    }
#pragma unroll
    for (int q = 0; q < TOPT; ++q) {
        ls[q] = rs[q];
        lj[q] = rj[q];
    }
}

// The slice's best TOPT (score, centroid id) of a warp's accumulators, written by lanes
// 0..TOPT-1 to part_s/part_j[o + lane]. Columns at or beyond ncols are ignored; col_ids
// maps a column to its centroid id (NULL: identity). Only columns that can be among them
// are sorted into the lanes' lists: with T the TOPT-th largest of the 32 lanes' maxima,
// TOPT columns (those maxima) score at least T, so every column of the result does too.
// Scores are non-negative and compare as their bit patterns. When fewer than TOPT lanes
// hold a positive score (T = 0), every column goes into the lists.
template <typename CT, int NV>
__device__ __forceinline__ void slice_topt_write(const float2 (&acc)[NV * 16 / (int)sizeof(CT) / 2], int64_t j0,
                                                 int lane, int32_t ncols, const int32_t *col_ids, float *part_s,
                                                 int32_t *part_j, int64_t o) {
    constexpr int EPV = 16 / (int)sizeof(CT);
    auto key_of = [&](int u, int e) -> uint32_t {
        const int64_t c = j0 + u * 32 * EPV + lane * EPV + e;
        const int qq = (u * EPV + e) >> 1;
        const float sc = (e & 1) ? acc[qq].y : acc[qq].x;
        return (c < ncols && sc > 0.f) ? __float_as_uint(sc) : 0u;
    };
    uint32_t mm = 0u;
#pragma unroll
    for (int u = 0; u < NV; ++u)
#pragma unroll
        for (int e = 0; e < EPV; ++e) mm = max(mm, key_of(u, e));
    uint32_t T = 0u;
#pragma unroll
    for (int q = 0; q < TOPT; ++q) {
        T = __reduce_max_sync(FULL, mm);
        const unsigned h = __ballot_sync(FULL, mm == T);
        if (lane == __ffs(h) - 1) mm = 0u;
    }
    float ls[TOPT];
    int lj[TOPT];
#pragma unroll
    for (int q = 0; q < TOPT; ++q) { ls[q] = -INFINITY; lj[q] = INT32_MAX; }
#pragma unroll
    for (int u = 0; u < NV; ++u) {
#pragma unroll
        for (int e = 0; e < EPV; ++e) {
            const int64_t c = j0 + u * 32 * EPV + lane * EPV + e;
            if (c < ncols && (T == 0u || key_of(u, e) >= T)) {
                const int id = col_ids ? __ldg(col_ids + c) : (int)c;
                const int qq = (u * EPV + e) >> 1;
                topt_insert(ls, lj, (e & 1) ? acc[qq].y : acc[qq].x, id);
            }
        }
    }
    topt_warp_select(ls, lj);
    if (lane < TOPT) {
        float sq = ls[0];
        int j = lj[0];
#pragma unroll
        for (int q = 1; q < TOPT; ++q) if (lane == q) { sq = ls[q]; j = lj[q]; }
        part_s[o + lane] = sq;
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
// u_c the unit roundoff of the centroid copy (0 for the FP32 master itself; 2^-8 for BF16
// round-to-nearest-even: an 8-bit significand, so a value just above a power of two can
// move by half of a 2^-7 spacing) and gamma_n = n u / (1 - n u), u = 2^-24, n = nonzeros
// of the document (one rounding per fused multiply-add). With a tensor-core head sum (BF16
// only) the head part's relative error, 2^-10 + 2^-11 + 2^-22 + (h / 16 + 2) 2^-22 at most
// (FP16 operands, FP16 stored sum, FP32 accumulation), is below u_c, and the sum enters the
// chain as one more term, which the head's own nonzeros outnumber: the same beta holds, plus
// the absolute term that the decision adds.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double score_beta(int precision, int64_t nnz) {
    const double u = 5.9604644775390625e-08;  // 2^-24
    const double nu = (double)nnz * u;
    const double gam = nu / (1.0 - nu);
    const double uc = precision == 1 ? 3.90625e-03 : 0.0;  // 2^-8
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
