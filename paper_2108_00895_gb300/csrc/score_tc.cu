// Head sums of the BF16 scoring pass on the tensor cores (the assignment step of Sec. 2; the
// pruned pass of Sec. 3.1 uses it unchanged on the compacted matrix).
//
// The collection's h most frequent terms (its head, chosen by document frequency) are dense
// across documents: in the Zipf collections the top 1024 terms carry close to half of the
// nonzeros at a density of several percent. For them the contraction X_head (documents x h)
// times C_head (h x columns) is a dense matrix product, computed here on the tensor cores;
// the remaining nonzeros (the tail) keep the warp-per-document gathers of the scoring
// kernel, which starts its accumulators from these head sums. Per document i and centroid j
//     s_ij = H_ij + sum over the tail nonzeros t of i, in CSR order, of x_it c_tj,
// H_ij = FP16(2^-20 times the tensor-core sum over the head terms of FP16(2^10 x_it) times
// FP16(2^10 c_tj)) (c from the FP32 master; exact products, FP32 accumulation in a fixed K
// order). Both parts depend only on (x_i, c_j) and the head set, which is fixed for a fit,
// so the full and the pruned pass still agree bit for bit.
//
// Error: |H_hat - H| <= (2^-10 + 2^-11 + 2^-22 + e_acc) H + 2^-34 (sum x + sum c) + 2^-25
// over the head terms: FP16 rounding of both operands, with the FP16 subnormal range (below
// 2^-24 in true scale) as an absolute term; e_acc = (h / 16 + 2) 2^-22 taken for the tensor
// core's FP32 accumulation of h / 16 steps of 16 exact products; the stored sum rounded to
// FP16 (2^-11 relative, 2^-25 absolute below 2^-14). The relative part is below the BF16
// copy's unit roundoff 2^-8, so the bound beta s of the plain BF16 pass still holds, and the
// absolute part, at most 2^-33 sqrt(nnz) + 2^-25, is added to the decision's threshold.
//
// Kernel k_head_gemm: persistent, one CTA of 10 warps per SM. A unit is 128 listed documents
// (one MMA tile, M = 128) x 256 columns (N = 256), accumulated over the h / 64 head blocks in
// one of two 256-column TMEM accumulators, so that the products of a unit overlap the
// draining of the previous one. Units are taken document tile by document tile, so a tile's
// rows stay in L2 across its column blocks. The document operand is the dense FP16 head
// matrix of the listed documents (k_head_rows, written once per scoring pass), the centroid
// operand the FP16 head matrix of the centroids; TMA brings both (128-byte swizzle, K-major).
// Warp roles:
//   - one thread issues the TMA copies of a stage (a 128 x 64 document box and a 256 x 64
//     centroid box);
//   - one thread issues the tcgen05.mma instructions (4 K-steps per block) into the unit's
//     accumulator and the commits that free a stage and announce a finished unit;
//   - 8 epilogue warps, 4 per accumulator (one per TMEM lane quarter), read the sums with
//     tcgen05.ld and store them, times 2^-20 and rounded to FP16, to out[position][column].
// Four stages overlap the loads of a block with the products of the previous ones. Every
// wait on an mbarrier is bounded: a timeout sets bit 32 of *err, skips the remaining work,
// waits (bounded) for the products and copies in flight and frees TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

#include "score_tc.cuh"
#include "skm_device.cuh"

namespace skm {

namespace {

constexpr int TC_M = 128;                       // documents per tile (MMA M, TMEM lanes)
constexpr int TC_KB = 64;                       // head terms per block (128 bytes of FP16)
constexpr int TC_N = 256;                       // columns per MMA
constexpr int A_BYTES = TC_M * TC_KB * 2;       // 16 KB
constexpr int B_HALF = TC_N * TC_KB * 2;        // 32 KB: one TMA box
constexpr int ERR_TC_TIMEOUT = 32;
constexpr long long WAIT_LIMIT = 1ll << 22;     // try_wait rounds before giving up


__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
// Bounded wait for the completion of the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(su32(b)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        :
        : "r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with the 128-byte swizzle (rows of 128
// bytes, 8-row groups 1024 bytes apart; the leading offset is unused for this layout).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5), FP16 A and B
// (bits 7-9, 10-12), both K-major (bits 15, 16), N / 8 (bits 17-22), M / 16 (bits 24-28).
constexpr uint32_t TC_IDESC =
    (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        :
        : "r"(tmem_d), "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(accumulate)
        : "memory");
}
// Arrive on bar once every tcgen05 operation this thread issued before has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 TMEM lanes x 16 columns: thread l of the warp receives lane (quarter base + l). The
// load is asynchronous: tmem_wait_ld() makes its registers valid.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Warp roles of k_head_gemm (10 warps): 0-7 epilogue (warp w reads TMEM lane quarter w % 4
// of accumulator w / 4), 8 issues the MMAs, 9 issues the TMA copies.
constexpr int HG_EPI_WARPS = 8;
constexpr int HG_MMA_WARP = 8;
constexpr int HG_TMA_WARP = 9;
constexpr int HG_WARPS = 10;
constexpr int HG_THREADS = HG_WARPS * 32;
constexpr int HG_DOCS = TC_M;                   // documents per unit: one MMA tile
constexpr int HG_STAGE = A_BYTES + B_HALF;      // one document tile + one 256-row centroid tile
constexpr int HG_STAGES = 4;
constexpr int HG_EPI_PER_BUF = HG_EPI_WARPS / 2;  // epilogue warps per TMEM accumulator
constexpr int HG_SMEM = HG_STAGES * HG_STAGE + 1024;
static_assert(HG_STAGE % 1024 == 0, "stages keep the 1024-byte swizzle alignment");

__global__ void __launch_bounds__(HG_THREADS, 1)
    k_head_gemm(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
                const HeadGemmArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                          ~static_cast<uintptr_t>(1023));
    __shared__ uint64_t full_s[HG_STAGES], empty_s[HG_STAGES], acc_full[2], acc_empty[2], end_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ uint32_t tma_g, mma_g;        // stage uses with copies issued / their arrival seen
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base_sh)),
                     "r"(2 * TC_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < HG_STAGES; ++s) {
            mbar_init(&full_s[s], 1);
            mbar_init(&empty_s[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], HG_EPI_PER_BUF);
        }
        mbar_init(&end_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_sh = 0;
        tma_g = 0;
        mma_g = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    const int kblocks = a.h / TC_KB;
    const int n_tiles = (a.n + HG_DOCS - 1) / HG_DOCS;
    const int n_units = n_tiles * a.n_cblk;

    if (warp == HG_TMA_WARP) {
        // ---- operands by TMA: stage g holds head block kb of the unit's document tile (rows
        // of the dense head matrix) and of its 256-column block of the centroid head
        if (lane == 0) {
            uint32_t g = 0;
            for (int u = blockIdx.x; u < n_units && !abort_sh; u += gridDim.x) {
                const int tile = u / a.n_cblk, cb = u - tile * a.n_cblk;
                for (int kb = 0; kb < kblocks; ++kb, ++g) {
                    const int s = g % HG_STAGES;
                    const uint32_t use = g / HG_STAGES;
                    if (use > 0 && !mbar_wait(&empty_s[s], (use - 1) & 1)) { abort_sh = 1; break; }
                    unsigned char *st = sm + s * HG_STAGE;
                    mbar_expect_tx(&full_s[s], HG_STAGE);
                    tma_load_2d(st, &amap, &full_s[s], kb * TC_KB, tile * HG_DOCS);
                    tma_load_2d(st + A_BYTES, &bmap, &full_s[s], kb * TC_KB, cb * TC_N);
                    tma_g = g + 1;
                }
            }
        }
    } else if (warp == HG_MMA_WARP) {
        // ---- products: per head block, 4 K-steps of M = 128, N = 256
        if (lane == 0) {
            uint32_t g = 0, v = 0;
            for (int u = blockIdx.x; u < n_units && !abort_sh; u += gridDim.x, ++v) {
                // accumulator v % 2, drained by its epilogue warps after its previous use
                const int ab = v & 1;
                if (v >= 2 && !mbar_wait(&acc_empty[ab], ((v >> 1) - 1) & 1)) { abort_sh = 1; break; }
                tc_fence_after();
                bool ok = true;
                for (int kb = 0; kb < kblocks; ++kb, ++g) {
                    const int s = g % HG_STAGES;
                    const uint32_t use = g / HG_STAGES;
                    if (!mbar_wait(&full_s[s], use & 1)) { ok = false; break; }
                    mma_g = g + 1;
                    tc_fence_after();
                    const uint32_t a0 = su32(sm + s * HG_STAGE), b0 = a0 + A_BYTES;
#pragma unroll
                    for (int ks = 0; ks < TC_KB / 16; ++ks)
                        tc_mma(tmem + ab * TC_N, sw128_desc(a0 + ks * 32), sw128_desc(b0 + ks * 32),
                               (kb | ks) != 0 ? 1u : 0u);
                    tc_commit(&empty_s[s]);
                }
                if (!ok) { abort_sh = 1; break; }
                tc_commit(&acc_full[ab]);
            }
        }
    } else {
        // ---- epilogue: TMEM -> head sums in global memory (times 2^-20, rounded to FP16)
        // warp w drains TMEM lane quarter w % 4 of accumulator w / 4: the CTA's units
        // v = w / 4, w / 4 + 2, ...
        const int q = warp & 3, ab = warp >> 2;
        uint32_t v = ab;
        for (int u = blockIdx.x + ab * gridDim.x; u < n_units && !abort_sh; u += 2 * gridDim.x, v += 2) {
            const int tile = u / a.n_cblk, cb = u - tile * a.n_cblk;
            const bool ok = mbar_wait(&acc_full[ab], (v >> 1) & 1);
            if (__any_sync(FULL, !ok)) { abort_sh = 1; break; }
            tc_fence_after();
            const int p = tile * HG_DOCS + 32 * q + lane;
            __half *dst = a.out + (int64_t)p * a.ld + (int64_t)cb * TC_N;
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ab * TC_N);
            constexpr float back = 1.0f / (TC_SCALE * TC_SCALE);   // 2^-20, exact
            // 64 columns per TMEM round trip: four loads in flight, one wait
            for (int c0 = 0; c0 < TC_N; c0 += 64) {
                uint32_t rr[64];
#pragma unroll
                for (int w4 = 0; w4 < 4; ++w4) tmem_ld16(taddr + (uint32_t)(c0 + 16 * w4), rr + 16 * w4);
                tmem_wait_ld();
                if (p < a.n) {
                    uint4 *d4 = reinterpret_cast<uint4 *>(dst + c0);
#pragma unroll
                    for (int w8 = 0; w8 < 8; ++w8) {
                        uint32_t hv[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const __half2 h2 = __floats2half2_rn(__uint_as_float(rr[8 * w8 + 2 * j]) * back,
                                                                 __uint_as_float(rr[8 * w8 + 2 * j + 1]) * back);
                            hv[j] = *reinterpret_cast<const uint32_t *>(&h2);
                        }
                        d4[w8] = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&acc_empty[ab])) : "memory");
        }
    }

    // ---- teardown: after a timeout, wait (bounded) for the products and the copies in
    // flight (the copies issued whose arrival no product waited for)
    __syncthreads();
    if (warp == HG_MMA_WARP && lane == 0 && abort_sh) {
        atomicOr(a.err, ERR_TC_TIMEOUT);
        tc_commit(&end_bar);                 // completes once every product issued completed
        mbar_wait(&end_bar, 0);
        for (uint32_t g = mma_g; g < tma_g; ++g)
            if (!mbar_wait(&full_s[g % HG_STAGES], (g / HG_STAGES) & 1)) break;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_N) : "memory");
    }
}

// Dense head rows of listed documents: X[p][q] = FP16 bits of 2^10 x of the head term at
// position q of the document at list position pos0 + p (0 elsewhere), for p < rows (rows at
// or beyond n stay 0). One warp per row, built in shared memory and stored with 16-byte
// writes.
constexpr int HR_WARPS = 8;
__global__ void __launch_bounds__(HR_WARPS * 32) k_head_rows(const int64_t *hptr, const uint32_t *hent,
                                                             const int32_t *doc_list, int32_t pos0, int32_t n,
                                                             int32_t rows, int32_t h, __half *X) {
    __shared__ __align__(16) uint16_t buf[HR_WARPS][TC_HEAD_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int p = blockIdx.x * HR_WARPS + w;
    if (p >= rows) return;
    uint4 *b4 = reinterpret_cast<uint4 *>(buf[w]);
    for (int c = lane; c < h / 8; c += 32) b4[c] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    if (p < n) {
        const int gp = pos0 + p;
        const int64_t i = doc_list ? (int64_t)doc_list[gp] : (int64_t)gp;
        const int64_t beg = hptr[i], end = hptr[i + 1];
        for (int64_t e = beg + lane; e < end; e += 32) {
            const uint32_t v = __ldg(hent + e);
            buf[w][v >> 16] = (uint16_t)(v & 0xffffu);
        }
    }
    __syncwarp();
    uint4 *dst = reinterpret_cast<uint4 *>(X + (int64_t)p * h);
    for (int c = lane; c < h / 8; c += 32) dst[c] = b4[c];
}

// ------------------------------------------------------------------------------------
// Head and tail split of a collection, head matrices
// ------------------------------------------------------------------------------------
__global__ void k_split_count(const int64_t *row_ptr, const int32_t *col, int64_t n, const int32_t *head_pos,
                              uint32_t *hcnt, uint32_t *tcnt) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int64_t beg = row_ptr[i], end = row_ptr[i + 1];
    uint32_t c = 0;
    for (int64_t p = beg + lane; p < end; p += 32) c += __ldg(head_pos + __ldg(col + p)) >= 0 ? 1u : 0u;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
    if (lane == 0) {
        hcnt[i] = c;
        tcnt[i] = (uint32_t)(end - beg) - c;
    }
}

// One warp per row: the head and tail entries keep their CSR order (warp-wide ballots).
__global__ void k_split_fill(const int64_t *row_ptr, const int32_t *col, const float *val, int64_t n,
                             const int32_t *head_pos, const int64_t *hptr, const int64_t *tptr, uint32_t *hent,
                             int32_t *tcol, float *tval) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int64_t beg = row_ptr[i], end = row_ptr[i + 1];
    int64_t ho = hptr[i], to = tptr[i];
    const unsigned below = (1u << lane) - 1u;
    for (int64_t b = beg; b < end; b += 32) {
        const int64_t p = b + lane;
        const bool in = p < end;
        const int32_t t = in ? __ldg(col + p) : 0;
        const float x = in ? __ldg(val + p) : 0.f;
        const int32_t hp = in ? __ldg(head_pos + t) : -1;
        const bool is_h = in && hp >= 0;
        const unsigned mh = __ballot_sync(FULL, is_h);
        const unsigned mt = __ballot_sync(FULL, in && !is_h);
        if (is_h) {
            const __half xh = __float2half_rn(x * TC_SCALE);
            hent[ho + __popc(mh & below)] = ((uint32_t)hp << 16) | (uint32_t)__half_as_ushort(xh);
        } else if (in) {
            const int64_t o = to + __popc(mt & below);
            tcol[o] = t;
            tval[o] = x;
        }
        ho += __popc(mh);
        to += __popc(mt);
    }
}

// headT[r * h + q] = FP16(2^10 C32[H[q] * ldc + col(r)]): 32 x 32 tiles through shared
// memory, reads along the centroid row (columns r), writes along the head position q.
__global__ void k_head_matrix(const float *C32, int64_t ldc, const int32_t *H, int32_t h, const int32_t *cols,
                              int32_t ncols, int64_t rows, __half *headT) {
    __shared__ float t[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int q0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int yy = ty; yy < 32; yy += 8) {
        const int q = q0 + yy;
        const int64_t r = r0 + tx;
        float v = 0.f;
        if (q < h && r < ncols) v = C32[(int64_t)H[q] * ldc + (cols ? (int64_t)cols[r] : r)];
        t[yy][tx] = v;
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        const int64_t r = r0 + yy;
        const int q = q0 + tx;
        if (r < rows && q < h) headT[r * h + q] = __float2half_rn(t[tx][yy] * TC_SCALE);
    }
}

std::once_flag g_encode_once;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

}  // namespace

cudaError_t tc_make_map(const __half *headT, int32_t h, int64_t rows, int32_t box_rows, CUtensorMap *out) {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) return cudaErrorNotSupported;
    if (h <= 0 || h % TC_KB != 0 || (box_rows != TC_M && box_rows != TC_N) || rows < box_rows ||
        (reinterpret_cast<uintptr_t>(headT) & 15) != 0)
        return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {(cuuint64_t)h, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)h * sizeof(__half)};
    const cuuint32_t box[2] = {(cuuint32_t)TC_KB, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = g_encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half *>(headT), dims, strides,
                                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_head_rows(const HeadGemmArgs &a, int32_t rows, __half *X, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    if (a.h <= 0 || a.h % TC_KB != 0 || a.h > TC_HEAD_MAX) return cudaErrorInvalidValue;
    k_head_rows<<<(unsigned)((rows + HR_WARPS - 1) / HR_WARPS), HR_WARPS * 32, 0, st>>>(a.hptr, a.hent, a.doc_list,
                                                                                      a.pos0, a.n, rows, a.h, X);
    return cudaGetLastError();
}

cudaError_t launch_head_gemm(const HeadGemmArgs &a, const CUtensorMap &amap, const CUtensorMap &bmap,
                             cudaStream_t st) {
    if (a.n <= 0 || a.n_cblk <= 0) return cudaSuccess;
    if (a.h <= 0 || a.h % TC_KB != 0 || a.h > TC_HEAD_MAX || a.ld < (int64_t)a.n_cblk * TC_N)
        return cudaErrorInvalidValue;
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_head_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, HG_SMEM);
    if (e != cudaSuccess) return e;
    const int64_t n_units = (int64_t)((a.n + HG_DOCS - 1) / HG_DOCS) * a.n_cblk;
    const unsigned grid = (unsigned)std::min<int64_t>(n_units, n_sm > 0 ? n_sm : 1);
    k_head_gemm<<<grid, HG_THREADS, HG_SMEM, st>>>(amap, bmap, a);
    return cudaGetLastError();
}

cudaError_t launch_split_count(const int64_t *row_ptr, const int32_t *col, int64_t n, const int32_t *head_pos,
                               uint32_t *hcnt, uint32_t *tcnt, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_split_count<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(row_ptr, col, n, head_pos, hcnt, tcnt);
    return cudaGetLastError();
}

cudaError_t launch_split_fill(const int64_t *row_ptr, const int32_t *col, const float *val, int64_t n,
                              const int32_t *head_pos, const int64_t *hptr, const int64_t *tptr, uint32_t *hent,
                              int32_t *tcol, float *tval, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_split_fill<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(row_ptr, col, val, n, head_pos, hptr, tptr, hent,
                                                                   tcol, tval);
    return cudaGetLastError();
}

cudaError_t launch_head_matrix(const float *C32, int64_t ldc, const int32_t *H, int32_t h, const int32_t *cols,
                               int32_t ncols, int64_t rows, __half *headT, cudaStream_t st) {
    if (rows <= 0 || h <= 0) return cudaSuccess;
    dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((h + 31) / 32));
    k_head_matrix<<<grid, dim3(32, 8), 0, st>>>(C32, ldc, H, h, cols, ncols, rows, headT);
    return cudaGetLastError();
}

}  // namespace skm
