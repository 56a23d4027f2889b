// C ABI of libskm (declared in include/skm.h): context, device memory, and the host side of
// the Lloyd loop (Sec. 2 of the paper) with the non-changing-clusters skip (Sec. 3.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "score_tc.cuh"
#include "skm.h"
#include "skm_host.h"
#include "skm_kernels.cuh"

using namespace skm;

namespace {

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct skm_ctx {
    skm_config cfg{};
    cudaStream_t st = nullptr;
    std::string err;
    size_t used = 0;
    std::vector<Buf *> owned;

    // resident centroids
    int32_t d = 0;
    int64_t ldc = 0;
    int slice = 0;
    Buf C32, C16, CM, norm_store, sq_store;

    // staged documents (host inputs are copied here)
    Buf d_row_ptr, d_col, d_val;
    // transposed postings
    Buf col_ptr, row_idx, cval, pterm, tcount, light_t0, light_t1, heavy_terms;
    Buf vh_terms, vch_h, vch_p0, vch_p1, vh_sum;   // very frequent terms, split into chunks
    // per-document state
    Buf abuf[2], s_state, r_state, clean, mdoc, order, order_hist;
    Buf part_s, part_j;
    Buf list_a, list_b, rs_doc, rs_cand, refull, full64, collect_doc, collect_thr, cand, cand_cnt;
    // per-cluster state
    Buf changed, sizes, moved, pos_in_m, normsq, inv_norm, dot_fx, newsq;
    Buf normsq128, sq128;
    Buf counters, counters64, scal, obj, init_ids;
    int32_t *h_counters = nullptr;  // pinned mirror
    unsigned long long *h_counters64 = nullptr;
    double *h_scal = nullptr;

    // sparse-row index of the scoring matrices (C, and CM for the pruned pass): rows of C with
    // at most k / rare_div nonzeros; cent_epoch counts centroid changes, docs_epoch stagings
    Buf rflag, rtot, rbase, rptr_c, rent_c, rptr_m, rent_m, colm, skipped;
    int rare_div = 0;
    int64_t cent_epoch = 1, docs_epoch = 0;
    int64_t rare_c_epoch = 0, rare_m_epoch = 0, colm_epoch = 0, colm_docs = -1;
    int32_t rare_m_ncols = -1;
    int64_t rare_c_rows = 0, rare_c_entries = 0;
    std::vector<uint32_t> h_rtot;

    // support of each centroid column, known on the host (fit only): 0 = the terms of its
    // current members, 1 = the terms of its seed document, 2 = unknown (cleared densely)
    std::vector<uint8_t> csupport;
    std::vector<uint8_t> h_changed;
    std::vector<int32_t> h_sizes, h_list;
    std::vector<uint8_t> h_flag;
    Buf zflag, zlist;
    bool cm_valid = false;   // the compacted moved matrix matches the last moved list
    // k-means++ seeding
    Buf pp_dist, pp_w, pp_csum, pp_drawn, pp_seed, pp_ids, pp_u;
    // threshold index of Sec. 3.2 (tindex.cu), built for centroid epoch ti_epoch
    Buf ti_G, ti_gcnt, ti_gptr, ti_hist, ti_mtab, ti_P, ti_pbe, ti_stats, ti_dump, ti_scan;
    int64_t ti_epoch = 0, ti_nzC = 0;
    // G and the value bins describe the centroids of epoch ti_maint_epoch; the update keeps
    // them current (clearing and setting the bits and counts of the entries it rewrites)
    int64_t ti_maint_epoch = -1;

    // tensor-core head of the BF16 scoring pass (score_tc.cu): the head set (chosen by
    // document frequency when a fit starts, or by the first assignment on loaded centroids),
    // the staged documents split into head entries and the tail CSR, and the FP16 head
    // matrices of the full and of the compacted centroid matrix with their TMA maps
    int32_t tc_h = 0;                 // head terms; 0: the head path is off
    int32_t tc_d = 0;                 // vocabulary the head set was chosen for
    int64_t tc_set = 0;               // bumps whenever the head set changes
    int64_t tc_nnz_head = 0;          // head nonzeros of the current split
    Buf tc_head_pos, tc_H, tc_df;
    Buf tc_hcnt, tc_tcnt, tc_hptr, tc_tptr, tc_hent, tc_tcol, tc_tval, tc_scan;
    int64_t tc_split_docs = -1, tc_split_set = -1;
    Buf tc_headT, tc_headMT, tc_hs, tc_X, tc_tcolm;
    int64_t tc_colm_epoch = -1, tc_colm_split = -1, tc_colm_set = -1;
    CUtensorMap tc_mapX{};
    const void *tc_mapX_ptr = nullptr;
    int32_t tc_mapX_h = 0;
    int64_t tc_mapX_rows = 0;
    CUtensorMap tc_mapT{}, tc_mapMT{};
    const void *tc_mapT_ptr = nullptr, *tc_mapMT_ptr = nullptr;
    int32_t tc_mapT_h = 0, tc_mapMT_h = 0;
    int64_t tc_T_epoch = -1, tc_T_set = -1, tc_MT_epoch = -1, tc_MT_set = -1;
    int32_t tc_MT_cols = -1;

    skm_stats stats{};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_score, ev_decide, ev_update, ev_index, ev_query, ev_head;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_next = 0;
};

namespace {

constexpr int kCollectCap = 64;          // candidates kept per document by the collect pass
constexpr int64_t kCollectBatch = 65536; // documents per collect launch

skm_status fail(skm_ctx *c, skm_status s, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
skm_status fail(skm_ctx *c, skm_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
    return s;
}

#define SKM_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(ctx, SKM_ERR_CUDA, "%s failed: %s (%s:%d)", #call,                 \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                       \
    } while (0)

#define SKM_TRY(expr)                  \
    do {                               \
        skm_status s_ = (expr);        \
        if (s_ != SKM_OK) return s_;   \
    } while (0)

void release(skm_ctx *ctx, Buf &b) {
    if (!b.p) return;
    if (ctx->cfg.free) ctx->cfg.free(b.p, b.bytes, ctx->cfg.alloc_user);
    else cudaFree(b.p);
    ctx->used -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
}

// Grow-only allocation; contents are not preserved when the buffer grows.
skm_status ensure(skm_ctx *ctx, Buf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    if (b.bytes >= bytes) return SKM_OK;
    const size_t old = b.bytes;
    if (ctx->cfg.mem_budget && ctx->used - old + bytes > ctx->cfg.mem_budget)
        return fail(ctx, SKM_ERR_BUDGET, "device memory budget exceeded: %zu + %zu > %zu bytes",
                    ctx->used - old, bytes, ctx->cfg.mem_budget);
    release(ctx, b);
    void *p = nullptr;
    if (ctx->cfg.alloc) {
        p = ctx->cfg.alloc(bytes, ctx->cfg.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (!p) return fail(ctx, SKM_ERR_OOM, "device allocation of %zu bytes failed", bytes);
    b.p = p;
    b.bytes = bytes;
    ctx->used += bytes;
    return SKM_OK;
}

template <typename T>
T *P(Buf &b) { return reinterpret_cast<T *>(b.p); }

// ---------------------------------------------------------------- timing
cudaEvent_t next_event(skm_ctx *ctx) {
    if (ctx->ev_next == ctx->ev_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        ctx->ev_pool.push_back(e);
    }
    return ctx->ev_pool[ctx->ev_next++];
}

struct Timed {
    skm_ctx *ctx;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *v;
    cudaEvent_t b = nullptr;
    Timed(skm_ctx *c, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &vec) : ctx(c), v(&vec) {
        if (ctx->cfg.timing) {
            b = next_event(ctx);
            cudaEventRecord(b, ctx->st);
        }
    }
    ~Timed() {
        if (b) {
            cudaEvent_t e = next_event(ctx);
            cudaEventRecord(e, ctx->st);
            v->emplace_back(b, e);
        }
    }
};

void collect_times(skm_ctx *ctx) {
    auto sum = [](std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &v) {
        double ms = 0;
        for (auto &pr : v) {
            float t = 0;
            if (cudaEventElapsedTime(&t, pr.first, pr.second) == cudaSuccess) ms += t;
        }
        v.clear();
        return ms;
    };
    ctx->stats.ms_score += sum(ctx->ev_score);
    ctx->stats.ms_decide += sum(ctx->ev_decide);
    ctx->stats.ms_update += sum(ctx->ev_update);
    ctx->stats.ms_index += sum(ctx->ev_index);
    ctx->stats.ms_query += sum(ctx->ev_query);
    ctx->stats.ms_head += sum(ctx->ev_head);
    ctx->ev_next = 0;
}

// ---------------------------------------------------------------- helpers
skm_status sync(skm_ctx *ctx) {
    SKM_CUDA(cudaStreamSynchronize(ctx->st));
    return SKM_OK;
}

skm_status read_counters(skm_ctx *ctx) {
    SKM_CUDA(cudaMemcpyAsync(ctx->h_counters, ctx->counters.p, CNT_N * sizeof(int32_t),
                             cudaMemcpyDeviceToHost, ctx->st));
    SKM_CUDA(cudaMemcpyAsync(ctx->h_counters64, ctx->counters64.p, C64_N * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, ctx->st));
    return sync(ctx);
}

skm_status reset_counters(skm_ctx *ctx) {
    SKM_CUDA(cudaMemsetAsync(ctx->counters.p, 0, CNT_N * sizeof(int32_t), ctx->st));
    SKM_CUDA(cudaMemsetAsync(ctx->counters64.p, 0, C64_N * sizeof(unsigned long long), ctx->st));
    return SKM_OK;
}

// Partial counts of the multiply-adds by exact zeros that sparse rows skip.
skm_status reset_skipped(skm_ctx *ctx) {
    SKM_TRY(ensure(ctx, ctx->skipped, sizeof(unsigned long long) * SKIP_COUNTERS));
    SKM_CUDA(cudaMemsetAsync(ctx->skipped.p, 0, sizeof(unsigned long long) * SKIP_COUNTERS, ctx->st));
    return SKM_OK;
}

skm_status read_skipped(skm_ctx *ctx, int64_t *out) {
    unsigned long long h[SKIP_COUNTERS];
    SKM_CUDA(cudaMemcpyAsync(h, ctx->skipped.p, sizeof h, cudaMemcpyDeviceToHost, ctx->st));
    SKM_TRY(sync(ctx));
    unsigned long long t = 0;
    for (unsigned long long v : h) t += v;
    *out = (int64_t)t;
    return SKM_OK;
}

struct DevCsr {
    int64_t n;
    int32_t d;
    int64_t nnz;
    const int64_t *row_ptr;
    const int32_t *col;
    const float *val;
};

// Host checks, staging (copy of host inputs), and device validation.
skm_status stage_docs(skm_ctx *ctx, const skm_csr *docs, DevCsr &out) {
    if (!docs) return fail(ctx, SKM_ERR_INVALID, "docs is NULL");
    if (docs->n_docs < 1) return fail(ctx, SKM_ERR_INVALID, "n_docs must be >= 1");
    if (docs->n_docs > INT32_MAX - 1) return fail(ctx, SKM_ERR_INVALID, "n_docs too large");
    if (docs->n_terms < 1) return fail(ctx, SKM_ERR_INVALID, "n_terms must be >= 1");
    if (docs->nnz < docs->n_docs) return fail(ctx, SKM_ERR_INVALID, "nnz < n_docs: empty rows");
    if (!docs->row_ptr || !docs->col_idx || !docs->values)
        return fail(ctx, SKM_ERR_INVALID, "NULL CSR array");
    out.n = docs->n_docs;
    out.d = docs->n_terms;
    out.nnz = docs->nnz;
    ctx->docs_epoch++;
    if (docs->on_device) {
        int64_t ends[2];
        SKM_CUDA(cudaMemcpyAsync(&ends[0], docs->row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->st));
        SKM_CUDA(cudaMemcpyAsync(&ends[1], docs->row_ptr + docs->n_docs, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, ctx->st));
        SKM_TRY(sync(ctx));
        if (ends[0] != 0 || ends[1] != docs->nnz)
            return fail(ctx, SKM_ERR_INVALID, "row_ptr[0] must be 0 and row_ptr[n_docs] == nnz");
        out.row_ptr = docs->row_ptr;
        out.col = docs->col_idx;
        out.val = docs->values;
    } else {
        if (docs->row_ptr[0] != 0 || docs->row_ptr[docs->n_docs] != docs->nnz)
            return fail(ctx, SKM_ERR_INVALID, "row_ptr[0] must be 0 and row_ptr[n_docs] == nnz");
        SKM_TRY(ensure(ctx, ctx->d_row_ptr, sizeof(int64_t) * (docs->n_docs + 1)));
        SKM_TRY(ensure(ctx, ctx->d_col, sizeof(int32_t) * docs->nnz));
        SKM_TRY(ensure(ctx, ctx->d_val, sizeof(float) * docs->nnz));
        SKM_CUDA(cudaMemcpyAsync(ctx->d_row_ptr.p, docs->row_ptr, sizeof(int64_t) * (docs->n_docs + 1),
                                 cudaMemcpyHostToDevice, ctx->st));
        SKM_CUDA(cudaMemcpyAsync(ctx->d_col.p, docs->col_idx, sizeof(int32_t) * docs->nnz,
                                 cudaMemcpyHostToDevice, ctx->st));
        SKM_CUDA(cudaMemcpyAsync(ctx->d_val.p, docs->values, sizeof(float) * docs->nnz,
                                 cudaMemcpyHostToDevice, ctx->st));
        out.row_ptr = P<int64_t>(ctx->d_row_ptr);
        out.col = P<int32_t>(ctx->d_col);
        out.val = P<float>(ctx->d_val);
    }
    SKM_TRY(reset_counters(ctx));
    SKM_CUDA(launch_validate(out.row_ptr, out.col, out.val, out.n, out.nnz, out.d,
                             P<int32_t>(ctx->counters) + CNT_ERR, ctx->st));
    ctx->stats.launches_total++;
    SKM_TRY(read_counters(ctx));
    const int e = ctx->h_counters[CNT_ERR];
    if (e) {
        std::string why;
        if (e & 1) why += " column index out of range or not strictly increasing;";
        if (e & 2) why += " value negative or not finite;";
        if (e & 4) why += " empty row;";
        if (e & 8) why += " row L2 norm not within 1e-5 of 1;";
        if (e & 16) why += " row offsets outside [0, nnz] or decreasing;";
        return fail(ctx, SKM_ERR_INVALID, "invalid documents:%s", why.c_str());
    }
    return SKM_OK;
}

// Resident centroid matrices for vocabulary size d (contents zeroed when (re)allocated). The
// compacted moved-centroid matrix is needed only by the Lloyd loop and the update (with_cm);
// a context that only assigns against loaded centroids does not hold it.
skm_status ensure_centroids(skm_ctx *ctx, int32_t d, bool zero, bool with_cm) {
    const int32_t k = ctx->cfg.k;
    const size_t n = (size_t)d * (size_t)ctx->ldc;
    const size_t cm_bytes = n * (ctx->cfg.precision == SKM_BF16 ? 2 : 4);
    const bool fresh = ctx->d != d || !ctx->C32.p;
    SKM_TRY(ensure(ctx, ctx->C32, n * sizeof(float)));
    if (ctx->cfg.precision == SKM_BF16) SKM_TRY(ensure(ctx, ctx->C16, n * sizeof(__nv_bfloat16)));
    const void *cm_before = ctx->CM.p;
    if (with_cm) SKM_TRY(ensure(ctx, ctx->CM, cm_bytes));
    SKM_TRY(ensure(ctx, ctx->norm_store, sizeof(double) * k));
    SKM_TRY(ensure(ctx, ctx->sq_store, sizeof(double) * k));
    if (fresh || zero) {
        SKM_CUDA(cudaMemsetAsync(ctx->C32.p, 0, n * sizeof(float), ctx->st));
        if (ctx->C16.p) SKM_CUDA(cudaMemsetAsync(ctx->C16.p, 0, n * sizeof(__nv_bfloat16), ctx->st));
        SKM_CUDA(cudaMemsetAsync(ctx->norm_store.p, 0, sizeof(double) * k, ctx->st));
        SKM_CUDA(cudaMemsetAsync(ctx->sq_store.p, 0, sizeof(double) * k, ctx->st));
    }
    if (with_cm && (fresh || zero || ctx->CM.p != cm_before))
        SKM_CUDA(cudaMemsetAsync(ctx->CM.p, 0, cm_bytes, ctx->st));
    ctx->d = d;
    ctx->cent_epoch++;
    return SKM_OK;
}

// Per-cluster buffers.
skm_status ensure_cluster_bufs(skm_ctx *ctx) {
    const int32_t k = ctx->cfg.k;
    SKM_TRY(ensure(ctx, ctx->changed, k));
    SKM_TRY(ensure(ctx, ctx->sizes, sizeof(int32_t) * k));
    SKM_TRY(ensure(ctx, ctx->moved, sizeof(int32_t) * k));
    SKM_TRY(ensure(ctx, ctx->pos_in_m, sizeof(int32_t) * k));
    SKM_TRY(ensure(ctx, ctx->normsq, sizeof(double) * k));
    SKM_TRY(ensure(ctx, ctx->inv_norm, sizeof(double) * k));
    SKM_TRY(ensure(ctx, ctx->dot_fx, sizeof(unsigned long long) * k));
    SKM_TRY(ensure(ctx, ctx->newsq, sizeof(double) * k));
    return SKM_OK;
}

// Per-document buffers for n documents.
skm_status ensure_doc_bufs(skm_ctx *ctx, int64_t n) {
    const int32_t k = ctx->cfg.k;
    const int64_t n_slices = (k + ctx->slice - 1) / ctx->slice;
    SKM_TRY(ensure(ctx, ctx->abuf[0], sizeof(int32_t) * n));
    SKM_TRY(ensure(ctx, ctx->abuf[1], sizeof(int32_t) * n));
    SKM_TRY(ensure(ctx, ctx->s_state, sizeof(float) * n));
    SKM_TRY(ensure(ctx, ctx->r_state, sizeof(float) * n));
    SKM_TRY(ensure(ctx, ctx->clean, n));
    SKM_TRY(ensure(ctx, ctx->mdoc, sizeof(int32_t) * n));
    SKM_TRY(ensure(ctx, ctx->order, sizeof(int32_t) * n));
    SKM_TRY(ensure(ctx, ctx->order_hist, sizeof(int32_t) * 4096));
    SKM_TRY(ensure(ctx, ctx->part_s, sizeof(float) * n * n_slices * TOPT));
    SKM_TRY(ensure(ctx, ctx->part_j, sizeof(int32_t) * n * n_slices * TOPT));
    SKM_TRY(ensure(ctx, ctx->list_a, sizeof(int32_t) * n));
    SKM_TRY(ensure(ctx, ctx->list_b, sizeof(int32_t) * n));
    SKM_TRY(ensure(ctx, ctx->rs_doc, sizeof(int32_t) * n));
    SKM_TRY(ensure(ctx, ctx->rs_cand, sizeof(int32_t) * n * TOPT));
    SKM_TRY(ensure(ctx, ctx->refull, sizeof(int32_t) * n));
    SKM_TRY(ensure(ctx, ctx->full64, sizeof(int32_t) * n));
    SKM_TRY(ensure(ctx, ctx->collect_doc, sizeof(int32_t) * n));
    SKM_TRY(ensure(ctx, ctx->collect_thr, sizeof(float) * n));
    SKM_TRY(ensure(ctx, ctx->cand, sizeof(int32_t) * (size_t)std::min<int64_t>(n, kCollectBatch) * kCollectCap));
    SKM_TRY(ensure(ctx, ctx->cand_cnt, sizeof(int32_t) * (size_t)std::min<int64_t>(n, kCollectBatch)));
    return SKM_OK;
}

// Term-major postings of the staged documents and the update work lists.
struct Postings {
    int32_t n_light = 0;   // chunks of consecutive light terms
    int32_t n_heavy = 0;   // terms with more postings than a chunk holds
    int32_t n_vh = 0;      // of those, the very frequent terms summed in chunks
    int32_t n_vch = 0;     // their chunks
    int F = 0;             // fixed-point bits of the update sums
    int64_t d_eff = 0;     // terms with at least one posting
};

skm_status build_postings(skm_ctx *ctx, const DevCsr &dc, Postings &pg) {
    const int32_t d = dc.d;
    const int32_t k = ctx->cfg.k;
    SKM_TRY(ensure(ctx, ctx->tcount, sizeof(int32_t) * (d + 1)));
    SKM_TRY(ensure(ctx, ctx->col_ptr, sizeof(int64_t) * (d + 1)));
    SKM_TRY(ensure(ctx, ctx->row_idx, sizeof(int32_t) * dc.nnz));
    SKM_TRY(ensure(ctx, ctx->cval, sizeof(float) * dc.nnz));
    SKM_TRY(ensure(ctx, ctx->pterm, sizeof(int32_t) * dc.nnz));
    SKM_CUDA(cudaMemsetAsync(ctx->tcount.p, 0, sizeof(int32_t) * (d + 1), ctx->st));
    SKM_CUDA(launch_term_count(dc.col, dc.nnz, P<int32_t>(ctx->tcount), ctx->st));
    ctx->stats.launches_total++;
    std::vector<int32_t> cnt(d);
    SKM_CUDA(cudaMemcpyAsync(cnt.data(), ctx->tcount.p, sizeof(int32_t) * d, cudaMemcpyDeviceToHost, ctx->st));
    SKM_TRY(sync(ctx));
    std::vector<int64_t> cp(d + 1);
    cp[0] = 0;
    pg.d_eff = 0;
    for (int32_t t = 0; t < d; ++t) {
        cp[t + 1] = cp[t] + cnt[t];
        pg.d_eff += cnt[t] > 0;
    }
    // Fixed point: a posting value is at most 1 + 1e-5 and a sum has at most N of them, so
    // with 2^bits > N every sum stays below 2^62 and ||S||^2 below 2^124.
    int bits = 0;
    while ((int64_t(1) << bits) < dc.n + 1) ++bits;
    pg.F = 61 - bits;
    // light chunks: consecutive terms with at most `chunk` postings in all; the term span of a
    // chunk is capped so that (term offset, moved position) packs into 32 bits
    const int64_t chunk = update_chunk_postings();
    const int64_t span_cap = std::max<int64_t>(1, std::min<int64_t>(4096, (int64_t(0xffffffff) / std::max(k, 1))));
    std::vector<int32_t> l0, l1, heavy;
    int64_t w = 0;
    int32_t start = -1, last = -1;
    auto close = [&](int32_t end) {
        if (start >= 0) {
            l0.push_back(start);
            l1.push_back(end);
        }
        start = -1;
        w = 0;
    };
    // very frequent terms go to the split path, most frequent first, as long as their sums
    // (one 64-bit integer per moved cluster) fit in 512 MB
    std::vector<int32_t> by_count;
    for (int32_t t = 0; t < d; ++t)
        if (cnt[t] > update_vh_postings()) by_count.push_back(t);
    std::sort(by_count.begin(), by_count.end(), [&](int32_t x, int32_t y) { return cnt[x] > cnt[y] || (cnt[x] == cnt[y] && x < y); });
    const size_t vh_cap = (size_t(512) << 20) / (sizeof(unsigned long long) * (size_t)std::max(k, 1));
    if (by_count.size() > vh_cap) by_count.resize(vh_cap);
    std::vector<uint8_t> is_vh(d, 0);
    for (int32_t t : by_count) is_vh[t] = 1;
    std::vector<int32_t> vh, vch_h;
    std::vector<int64_t> vch_p0, vch_p1;
    for (int32_t t = 0; t < d; ++t) {
        if (cnt[t] > chunk) {          // a chunk's posting range never spans a heavy term
            close(t);
            if (is_vh[t]) {
                const int32_t h = (int32_t)vh.size();
                vh.push_back(t);
                for (int64_t p = cp[t]; p < cp[t + 1]; p += update_vh_chunk()) {
                    vch_h.push_back(h);
                    vch_p0.push_back(p);
                    vch_p1.push_back(std::min<int64_t>(p + update_vh_chunk(), cp[t + 1]));
                }
            } else {
                heavy.push_back(t);
            }
            continue;
        }
        if (cnt[t] == 0) continue;
        if (start >= 0 && (w + cnt[t] > chunk || t - start >= span_cap)) close(t);
        if (start < 0) start = t;
        w += cnt[t];
        last = t;
    }
    if (start >= 0) close(last + 1);
    pg.n_light = (int32_t)l0.size();
    pg.n_heavy = (int32_t)heavy.size();
    pg.n_vh = (int32_t)vh.size();
    pg.n_vch = (int32_t)vch_h.size();
    if (pg.n_vh) {
        SKM_TRY(ensure(ctx, ctx->vh_terms, sizeof(int32_t) * pg.n_vh));
        SKM_TRY(ensure(ctx, ctx->vch_h, sizeof(int32_t) * pg.n_vch));
        SKM_TRY(ensure(ctx, ctx->vch_p0, sizeof(int64_t) * pg.n_vch));
        SKM_TRY(ensure(ctx, ctx->vch_p1, sizeof(int64_t) * pg.n_vch));
        SKM_TRY(ensure(ctx, ctx->vh_sum, sizeof(unsigned long long) * (size_t)pg.n_vh * k));
        SKM_CUDA(cudaMemcpyAsync(ctx->vh_terms.p, vh.data(), sizeof(int32_t) * pg.n_vh, cudaMemcpyHostToDevice, ctx->st));
        SKM_CUDA(cudaMemcpyAsync(ctx->vch_h.p, vch_h.data(), sizeof(int32_t) * pg.n_vch, cudaMemcpyHostToDevice, ctx->st));
        SKM_CUDA(cudaMemcpyAsync(ctx->vch_p0.p, vch_p0.data(), sizeof(int64_t) * pg.n_vch, cudaMemcpyHostToDevice, ctx->st));
        SKM_CUDA(cudaMemcpyAsync(ctx->vch_p1.p, vch_p1.data(), sizeof(int64_t) * pg.n_vch, cudaMemcpyHostToDevice, ctx->st));
    }
    SKM_TRY(ensure(ctx, ctx->light_t0, sizeof(int32_t) * std::max(pg.n_light, 1)));
    SKM_TRY(ensure(ctx, ctx->light_t1, sizeof(int32_t) * std::max(pg.n_light, 1)));
    SKM_TRY(ensure(ctx, ctx->heavy_terms, sizeof(int32_t) * std::max(pg.n_heavy, 1)));
    SKM_CUDA(cudaMemcpyAsync(ctx->col_ptr.p, cp.data(), sizeof(int64_t) * (d + 1), cudaMemcpyHostToDevice, ctx->st));
    if (pg.n_light)
        SKM_CUDA(cudaMemcpyAsync(ctx->light_t0.p, l0.data(), sizeof(int32_t) * pg.n_light, cudaMemcpyHostToDevice, ctx->st));
    if (pg.n_light)
        SKM_CUDA(cudaMemcpyAsync(ctx->light_t1.p, l1.data(), sizeof(int32_t) * pg.n_light, cudaMemcpyHostToDevice, ctx->st));
    if (pg.n_heavy)
        SKM_CUDA(cudaMemcpyAsync(ctx->heavy_terms.p, heavy.data(), sizeof(int32_t) * pg.n_heavy, cudaMemcpyHostToDevice, ctx->st));
    SKM_CUDA(cudaMemsetAsync(ctx->tcount.p, 0, sizeof(int32_t) * (d + 1), ctx->st));
    SKM_CUDA(launch_csc_fill(dc.row_ptr, dc.col, dc.val, dc.n, P<int64_t>(ctx->col_ptr), P<int32_t>(ctx->tcount),
                             P<int32_t>(ctx->row_idx), P<float>(ctx->cval), P<int32_t>(ctx->pterm), ctx->st));
    ctx->stats.launches_total++;
    SKM_TRY(ensure(ctx, ctx->normsq128, 2 * sizeof(unsigned long long) * k));
    SKM_TRY(ensure(ctx, ctx->sq128, 2 * sizeof(unsigned long long) * k));
    // the transient host vectors must outlive the async copies
    SKM_TRY(sync(ctx));
    return SKM_OK;
}

// Sparse rows of the scoring matrix of one pass (off: every row dense, plain column ids).
struct RareView {
    const int32_t *col = nullptr;   // column stream with sparse rows marked ~t
    const uint32_t *ptr = nullptr;
    const void *ent = nullptr;
    int32_t n_slices = 0;
};

// Builds, when stale, the sparse-row index of C (rows with at most k / rare_div nonzeros)
// and the marked column stream of the staged documents; for a pruned pass also the index
// of the compacted moved-centroid matrix CM over the same rows. The scores do not depend
// on which rows are sparse, so the index only has to describe the current matrices.
skm_status rare_index(skm_ctx *ctx, Buf &M, int32_t ncols, const uint8_t *only, bool classify, Buf &ptr, Buf &ent,
                      int64_t *rows_out, int64_t *entries_out) {
    const int32_t d = ctx->d;
    const int prec = ctx->cfg.precision;
    const int32_t S = (ncols + ctx->slice - 1) / ctx->slice;
    const uint32_t thr = (uint32_t)(ctx->cfg.k / std::max(ctx->rare_div, 1));
    SKM_TRY(ensure(ctx, ctx->rtot, sizeof(uint32_t) * d));
    SKM_TRY(ensure(ctx, ctx->rbase, sizeof(uint32_t) * d));
    SKM_TRY(ensure(ctx, ptr, sizeof(uint32_t) * (size_t)d * (S + 1)));
    SKM_CUDA(launch_rare_count(M.p, prec, ctx->ldc, d, ncols, ctx->slice, thr, only,
                               classify ? P<uint8_t>(ctx->rflag) : nullptr, P<uint32_t>(ctx->rtot), ctx->st));
    ctx->h_rtot.resize(d);
    SKM_CUDA(cudaMemcpyAsync(ctx->h_rtot.data(), ctx->rtot.p, sizeof(uint32_t) * d, cudaMemcpyDeviceToHost, ctx->st));
    SKM_TRY(sync(ctx));
    // exclusive scan on the host (d entries); the index uses 32-bit offsets
    uint64_t tot = 0;
    int64_t rows = 0;
    for (int32_t t = 0; t < d; ++t) {
        const uint32_t c = ctx->h_rtot[t];
        ctx->h_rtot[t] = (uint32_t)tot;
        tot += c;
        rows += c > 0;
        if (tot > 0xffffffffull) return fail(ctx, SKM_ERR_INVALID, "sparse-row index exceeds 2^32 entries");
    }
    const size_t esz = prec == SKM_BF16 ? 4 : 8;
    SKM_TRY(ensure(ctx, ent, esz * (size_t)std::max<uint64_t>(tot, 1)));
    SKM_CUDA(cudaMemcpyAsync(ctx->rbase.p, ctx->h_rtot.data(), sizeof(uint32_t) * d, cudaMemcpyHostToDevice, ctx->st));
    SKM_CUDA(launch_rare_fill(M.p, prec, ctx->ldc, d, ncols, ctx->slice, S, P<uint8_t>(ctx->rflag),
                              P<uint32_t>(ctx->rbase), P<uint32_t>(ptr), ent.p, ctx->st));
    SKM_TRY(sync(ctx));   // h_rtot is reused by the next build
    ctx->stats.launches_total += 2;
    if (rows_out) *rows_out = rows;
    if (entries_out) *entries_out = (int64_t)tot;
    return SKM_OK;
}

skm_status build_c_index(skm_ctx *ctx) {
    if (ctx->rare_div <= 0 || ctx->rare_c_epoch == ctx->cent_epoch) return SKM_OK;
    SKM_TRY(ensure(ctx, ctx->rflag, (size_t)ctx->d));
    Buf &C = ctx->cfg.precision == SKM_BF16 ? ctx->C16 : ctx->C32;
    SKM_TRY(rare_index(ctx, C, ctx->cfg.k, nullptr, true, ctx->rptr_c, ctx->rent_c, &ctx->rare_c_rows,
                       &ctx->rare_c_entries));
    ctx->rare_c_epoch = ctx->cent_epoch;
    ctx->rare_m_epoch = 0;
    return SKM_OK;
}

skm_status ensure_rare(skm_ctx *ctx, const DevCsr &dc, bool pruned, int32_t ncols, RareView &rv,
                       bool mark_collection = true) {
    rv = RareView{};
    if (ctx->rare_div <= 0) return SKM_OK;
    Timed tm(ctx, ctx->ev_index);
    SKM_TRY(build_c_index(ctx));
    if (mark_collection && (ctx->colm_epoch != ctx->rare_c_epoch || ctx->colm_docs != ctx->docs_epoch)) {
        SKM_TRY(ensure(ctx, ctx->colm, sizeof(int32_t) * (size_t)dc.nnz));
        SKM_CUDA(launch_mark_rare(dc.col, dc.nnz, P<uint8_t>(ctx->rflag), P<int32_t>(ctx->colm), ctx->st));
        ctx->stats.launches_total++;
        ctx->colm_epoch = ctx->rare_c_epoch;
        ctx->colm_docs = ctx->docs_epoch;
    }
    ctx->stats.sparse_rows = ctx->rare_c_rows;
    ctx->stats.sparse_entries = ctx->rare_c_entries;
    rv.col = P<int32_t>(ctx->colm);
    if (!pruned) {
        rv.ptr = P<uint32_t>(ctx->rptr_c);
        rv.ent = ctx->rent_c.p;
        rv.n_slices = (ctx->cfg.k + ctx->slice - 1) / ctx->slice;
        return SKM_OK;
    }
    if (ctx->rare_m_epoch != ctx->cent_epoch || ctx->rare_m_ncols != ncols) {
        SKM_TRY(rare_index(ctx, ctx->CM, ncols, P<uint8_t>(ctx->rflag), false, ctx->rptr_m, ctx->rent_m, nullptr,
                           nullptr));
        ctx->rare_m_epoch = ctx->cent_epoch;
        ctx->rare_m_ncols = ncols;
    }
    rv.ptr = P<uint32_t>(ctx->rptr_m);
    rv.ent = ctx->rent_m.p;
    rv.n_slices = (ncols + ctx->slice - 1) / ctx->slice;
    return SKM_OK;
}

// Points the pass at the marked column stream; returns the sparse rows (null: dense pass).
const SparseArgs *apply_rare(skm_ctx *ctx, const RareView &rv, ScoreArgs &sa, SparseArgs &sp) {
    if (!rv.ptr) return nullptr;
    sa.col = rv.col;
    sp.ptr = rv.ptr;
    sp.ent = rv.ent;
    sp.n_slices = rv.n_slices;
    sp.skipped = ctx->skipped.p ? P<unsigned long long>(ctx->skipped) : nullptr;
    return &sp;
}

// Scoring pass over a document list (nullable = all) against all k or the moved list,
// followed by the decision kernel.
// The threshold index's bitmap and value bins match the resident centroids.
bool ti_current(const skm_ctx *ctx) { return ctx->ti_G.p && ctx->ti_maint_epoch == ctx->cent_epoch; }

// Threshold index (Sec. 3.2) of the resident FP32 master, rebuilt when the centroids changed.
skm_status build_tindex(skm_ctx *ctx) {
    if (ctx->ti_epoch == ctx->cent_epoch) return SKM_OK;
    const int32_t k = ctx->cfg.k, d = ctx->d, W = ti_words(k);
    const int L = ctx->cfg.index_levels;
    Timed tm(ctx, ctx->ev_index);
    const size_t g_bytes = sizeof(uint32_t) * (size_t)d * W;
    const bool incremental = ti_current(ctx) && ctx->ti_G.bytes >= g_bytes;
    SKM_TRY(ensure(ctx, ctx->ti_G, g_bytes));
    SKM_TRY(ensure(ctx, ctx->ti_gcnt, sizeof(uint32_t) * (size_t)d));
    SKM_TRY(ensure(ctx, ctx->ti_gptr, sizeof(int64_t) * ((size_t)d + 1)));
    SKM_TRY(ensure(ctx, ctx->ti_hist, sizeof(uint32_t) * (size_t)k * TI_NB));
    SKM_TRY(ensure(ctx, ctx->ti_mtab, (size_t)L * k * TI_NB));
    SKM_TRY(ensure(ctx, ctx->ti_pbe, sizeof(uint32_t) * (size_t)L * d * TI_MB));
    if (incremental) {
        // the update kept G and the bins current: only the row counts are recounted
        SKM_CUDA(launch_ti_gcnt(P<uint32_t>(ctx->ti_G), d, W, P<uint32_t>(ctx->ti_gcnt), ctx->st));
    } else {
        SKM_CUDA(cudaMemsetAsync(ctx->ti_hist.p, 0, sizeof(uint32_t) * (size_t)k * TI_NB, ctx->st));
        SKM_CUDA(launch_ti_rows(P<float>(ctx->C32), ctx->ldc, d, k, P<uint32_t>(ctx->ti_G),
                                P<uint32_t>(ctx->ti_gcnt), P<uint32_t>(ctx->ti_hist), ctx->st));
    }
    SKM_TRY(ensure(ctx, ctx->ti_scan, ti_scan_scratch(d)));
    SKM_CUDA(launch_ti_scan(P<uint32_t>(ctx->ti_gcnt), d, P<int64_t>(ctx->ti_gptr), P<int64_t>(ctx->ti_scan), ctx->st));
    TiThr thr{};
    for (int l = 0; l < L; ++l) thr.v[l] = ctx->cfg.index_lambda[l] * ctx->cfg.index_lambda[l] * (1.0 - 1e-9);
    SKM_CUDA(launch_ti_mtab(P<uint32_t>(ctx->ti_hist), nullptr, k, k, L, thr, P<uint8_t>(ctx->ti_mtab), ctx->st));
    int64_t nz = 0;
    SKM_CUDA(cudaMemcpyAsync(&nz, P<int64_t>(ctx->ti_gptr) + d, sizeof nz, cudaMemcpyDeviceToHost, ctx->st));
    SKM_TRY(sync(ctx));
    ctx->ti_nzC = nz > 0 ? nz : 1;
    SKM_TRY(ensure(ctx, ctx->ti_P, sizeof(uint32_t) * (size_t)L * ctx->ti_nzC));
    SKM_CUDA(launch_ti_fill(P<float>(ctx->C32), ctx->ldc, d, k, P<uint32_t>(ctx->ti_G), P<uint8_t>(ctx->ti_mtab), L,
                            P<int64_t>(ctx->ti_gptr), ctx->ti_nzC, P<uint32_t>(ctx->ti_P), P<uint32_t>(ctx->ti_pbe),
                            ctx->st));
    ctx->stats.launches_total += 4;
    ctx->ti_epoch = ctx->cent_epoch;
    ctx->ti_maint_epoch = ctx->cent_epoch;
    return SKM_OK;
}

// Query arguments over the resident index (lists and state filled in by the caller).
TiQueryArgs ti_args(skm_ctx *ctx, const DevCsr &dc) {
    TiQueryArgs q{};
    q.row_ptr = dc.row_ptr;
    q.col = dc.col;
    q.val = dc.val;
    q.C32 = P<float>(ctx->C32);
    q.ldc = ctx->ldc;
    q.k = ctx->cfg.k;
    q.W = ti_words(ctx->cfg.k);
    q.d = ctx->d;
    q.G = P<uint32_t>(ctx->ti_G);
    q.P = P<uint32_t>(ctx->ti_P);
    q.nzC = ctx->ti_nzC;
    q.gptr = P<int64_t>(ctx->ti_gptr);
    q.pbe = P<uint32_t>(ctx->ti_pbe);
    q.L = ctx->cfg.index_levels;
    q.max_cands = ctx->cfg.index_max_cands;
    for (int l = 0; l < q.L; ++l) q.lam[l] = ctx->cfg.index_lambda[l];
    q.fixed_level = -1;
    return q;
}

// ---------------------------------------------------------------- tensor-core head
// The head path serves BF16 scoring with 512-column slices and dense rows.
bool tc_wanted(const skm_ctx *ctx) {
    return ctx->cfg.precision == SKM_BF16 && ctx->slice == TC_SLICE && ctx->ldc % TC_SLICE == 0 &&
           ctx->cfg.head_terms >= 0;
}

// Head set of the staged collection: the most frequent terms by document frequency (ties
// to the lower term id), kept in ascending term order so that a document's head entries
// come in CSR order. Automatic size: the terms in at least 1/64 of the documents, rounded
// down to a multiple of 64, between 64 and TC_HEAD_AUTO.
skm_status tc_choose_head(skm_ctx *ctx, const DevCsr &dc) {
    ctx->tc_h = 0;
    ctx->tc_d = 0;
    ctx->tc_set++;
    if (!tc_wanted(ctx) || dc.d < 64) return SKM_OK;
    Timed tm(ctx, ctx->ev_head);
    SKM_TRY(ensure(ctx, ctx->tc_df, sizeof(int32_t) * dc.d));
    SKM_CUDA(cudaMemsetAsync(ctx->tc_df.p, 0, sizeof(int32_t) * dc.d, ctx->st));
    SKM_CUDA(launch_term_count(dc.col, dc.nnz, P<int32_t>(ctx->tc_df), ctx->st));
    std::vector<int32_t> df(dc.d);
    SKM_CUDA(cudaMemcpyAsync(df.data(), ctx->tc_df.p, sizeof(int32_t) * dc.d, cudaMemcpyDeviceToHost, ctx->st));
    SKM_TRY(sync(ctx));
    const int32_t d64 = dc.d / 64 * 64;
    int32_t h = 0;
    if (ctx->cfg.head_terms > 0) {
        h = std::min(TC_HEAD_MAX, (ctx->cfg.head_terms + 63) / 64 * 64);
    } else {
        const int64_t min_df = std::max<int64_t>(1, (dc.n + 63) / 64);
        int64_t cnt = 0;
        for (int32_t v : df) cnt += v >= min_df;
        h = (int32_t)std::min<int64_t>(TC_HEAD_AUTO, std::max<int64_t>(64, cnt / 64 * 64));
    }
    h = std::min(h, d64);
    if (h < 64) return SKM_OK;
    std::vector<int32_t> idx(dc.d);
    for (int32_t t = 0; t < dc.d; ++t) idx[t] = t;
    auto more_frequent = [&](int32_t x, int32_t y) { return df[x] > df[y] || (df[x] == df[y] && x < y); };
    std::nth_element(idx.begin(), idx.begin() + (h - 1), idx.end(), more_frequent);
    std::vector<int32_t> H(idx.begin(), idx.begin() + h);
    std::sort(H.begin(), H.end());
    std::vector<int32_t> pos(dc.d, -1);
    for (int32_t q = 0; q < h; ++q) pos[H[q]] = q;
    SKM_TRY(ensure(ctx, ctx->tc_head_pos, sizeof(int32_t) * dc.d));
    SKM_TRY(ensure(ctx, ctx->tc_H, sizeof(int32_t) * h));
    SKM_CUDA(cudaMemcpyAsync(ctx->tc_head_pos.p, pos.data(), sizeof(int32_t) * dc.d, cudaMemcpyHostToDevice, ctx->st));
    SKM_CUDA(cudaMemcpyAsync(ctx->tc_H.p, H.data(), sizeof(int32_t) * h, cudaMemcpyHostToDevice, ctx->st));
    SKM_TRY(sync(ctx));
    ctx->tc_h = h;
    ctx->tc_d = dc.d;
    return SKM_OK;
}

// The staged collection split into the head entries and the tail CSR (current head set).
skm_status tc_split(skm_ctx *ctx, const DevCsr &dc) {
    if (ctx->tc_h == 0) return SKM_OK;
    if (ctx->tc_split_docs == ctx->docs_epoch && ctx->tc_split_set == ctx->tc_set) return SKM_OK;
    Timed tm(ctx, ctx->ev_head);
    const int64_t n = dc.n;
    SKM_TRY(ensure(ctx, ctx->tc_hcnt, sizeof(uint32_t) * n));
    SKM_TRY(ensure(ctx, ctx->tc_tcnt, sizeof(uint32_t) * n));
    SKM_TRY(ensure(ctx, ctx->tc_hptr, sizeof(int64_t) * (n + 1)));
    SKM_TRY(ensure(ctx, ctx->tc_tptr, sizeof(int64_t) * (n + 1)));
    SKM_TRY(ensure(ctx, ctx->tc_scan, ti_scan_scratch(n)));
    SKM_CUDA(launch_split_count(dc.row_ptr, dc.col, n, P<int32_t>(ctx->tc_head_pos), P<uint32_t>(ctx->tc_hcnt),
                                P<uint32_t>(ctx->tc_tcnt), ctx->st));
    SKM_CUDA(launch_ti_scan(P<uint32_t>(ctx->tc_hcnt), n, P<int64_t>(ctx->tc_hptr), P<int64_t>(ctx->tc_scan), ctx->st));
    SKM_CUDA(launch_ti_scan(P<uint32_t>(ctx->tc_tcnt), n, P<int64_t>(ctx->tc_tptr), P<int64_t>(ctx->tc_scan), ctx->st));
    int64_t tot[2] = {0, 0};
    SKM_CUDA(cudaMemcpyAsync(&tot[0], P<int64_t>(ctx->tc_hptr) + n, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->st));
    SKM_CUDA(cudaMemcpyAsync(&tot[1], P<int64_t>(ctx->tc_tptr) + n, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->st));
    SKM_TRY(sync(ctx));
    if (tot[0] + tot[1] != dc.nnz) return fail(ctx, SKM_ERR_CUDA, "head split lost entries");
    SKM_TRY(ensure(ctx, ctx->tc_hent, sizeof(uint32_t) * std::max<int64_t>(tot[0], 1)));
    SKM_TRY(ensure(ctx, ctx->tc_tcol, sizeof(int32_t) * std::max<int64_t>(tot[1], 1)));
    SKM_TRY(ensure(ctx, ctx->tc_tval, sizeof(float) * std::max<int64_t>(tot[1], 1)));
    SKM_CUDA(launch_split_fill(dc.row_ptr, dc.col, dc.val, n, P<int32_t>(ctx->tc_head_pos), P<int64_t>(ctx->tc_hptr),
                               P<int64_t>(ctx->tc_tptr), P<uint32_t>(ctx->tc_hent), P<int32_t>(ctx->tc_tcol),
                               P<float>(ctx->tc_tval), ctx->st));
    ctx->stats.launches_total += 4;
    ctx->tc_split_docs = ctx->docs_epoch;
    ctx->tc_split_set = ctx->tc_set;
    ctx->tc_nnz_head = tot[0];
    return SKM_OK;
}

// FP16 head matrix (2^10 C32 at the head rows, K-major) of the full matrix, or of the
// compacted matrix of the moved list, current for the resident centroids; its TMA map.
skm_status tc_matrix(skm_ctx *ctx, bool pruned, int32_t ncols, const CUtensorMap **map) {
    Buf &B = pruned ? ctx->tc_headMT : ctx->tc_headT;
    int64_t &epoch = pruned ? ctx->tc_MT_epoch : ctx->tc_T_epoch;
    int64_t &set = pruned ? ctx->tc_MT_set : ctx->tc_T_set;
    CUtensorMap &m = pruned ? ctx->tc_mapMT : ctx->tc_mapT;
    const void *&mp = pruned ? ctx->tc_mapMT_ptr : ctx->tc_mapT_ptr;
    int32_t &mh = pruned ? ctx->tc_mapMT_h : ctx->tc_mapT_h;
    const int64_t rows = ctx->ldc;
    const bool stale = epoch != ctx->cent_epoch || set != ctx->tc_set || (pruned && ctx->tc_MT_cols != ncols);
    if (stale) {
        Timed tm(ctx, ctx->ev_head);
        SKM_TRY(ensure(ctx, B, sizeof(__half) * (size_t)rows * ctx->tc_h));
        SKM_CUDA(launch_head_matrix(P<float>(ctx->C32), ctx->ldc, P<int32_t>(ctx->tc_H), ctx->tc_h,
                                    pruned ? P<int32_t>(ctx->moved) : nullptr, ncols, rows, P<__half>(B), ctx->st));
        ctx->stats.launches_total++;
        epoch = ctx->cent_epoch;
        set = ctx->tc_set;
        if (pruned) ctx->tc_MT_cols = ncols;
    }
    if (mp != B.p || mh != ctx->tc_h) {
        SKM_CUDA(tc_make_map(P<__half>(B), ctx->tc_h, rows, 256, &m));
        mp = B.p;
        mh = ctx->tc_h;
    }
    *map = &m;
    return SKM_OK;
}

bool tc_active(const skm_ctx *ctx) {
    return ctx->tc_h > 0 && tc_wanted(ctx) && ctx->tc_split_docs == ctx->docs_epoch && ctx->tc_split_set == ctx->tc_set;
}

// Scoring pass (or collect pass) with the tensor-core head: chunk by chunk of list
// positions, the head sums of the chunk (k_head_gemm, FP32 in a buffer of at most
// kHeadSumBytes) and then the scoring kernel over the tail nonzeros, starting from them.
constexpr int64_t kHeadSumBytes = int64_t(2) << 30;

skm_status tc_score(skm_ctx *ctx, const DevCsr &dc, const ScoreArgs &sa0, bool pruned, bool collect) {
    const CUtensorMap *map = nullptr;
    SKM_TRY(tc_matrix(ctx, pruned, sa0.ncols, &map));
    // sparse centroid rows (section 6a) over the tail: the tail's column stream marked the
    // same way as the full collection's
    RareView rv;
    SKM_TRY(ensure_rare(ctx, dc, pruned, sa0.ncols, rv, false));
    SparseArgs spa{};
    const SparseArgs *sp = nullptr;
    if (rv.ptr) {
        const int64_t n_tail = dc.nnz - ctx->tc_nnz_head;
        if (ctx->tc_colm_epoch != ctx->rare_c_epoch || ctx->tc_colm_split != ctx->tc_split_docs ||
            ctx->tc_colm_set != ctx->tc_set) {
            SKM_TRY(ensure(ctx, ctx->tc_tcolm, sizeof(int32_t) * (size_t)std::max<int64_t>(n_tail, 1)));
            SKM_CUDA(launch_mark_rare(P<int32_t>(ctx->tc_tcol), n_tail, P<uint8_t>(ctx->rflag),
                                      P<int32_t>(ctx->tc_tcolm), ctx->st));
            ctx->stats.launches_total++;
            ctx->tc_colm_epoch = ctx->rare_c_epoch;
            ctx->tc_colm_split = ctx->tc_split_docs;
            ctx->tc_colm_set = ctx->tc_set;
        }
        spa.ptr = rv.ptr;
        spa.ent = rv.ent;
        spa.n_slices = rv.n_slices;
        spa.skipped = ctx->skipped.p ? P<unsigned long long>(ctx->skipped) : nullptr;
        sp = &spa;
    }
    const int64_t ld = ctx->ldc;
    const int32_t n_slices = (sa0.ncols + TC_SLICE - 1) / TC_SLICE;
    int64_t cap_bytes = kHeadSumBytes;
    if (ctx->cfg.mem_budget) cap_bytes = std::min<int64_t>(cap_bytes, (int64_t)(ctx->cfg.mem_budget / 16));
    int64_t chunk = cap_bytes / (int64_t)(sizeof(__half) * ld) / 256 * 256;
    chunk = std::max<int64_t>(256, std::min<int64_t>(chunk, ((int64_t)sa0.n_list + 255) / 256 * 256));
    SKM_TRY(ensure(ctx, ctx->tc_hs, sizeof(__half) * (size_t)chunk * (size_t)ld));
    // dense head rows of a chunk's documents (the GEMM's document operand) and their TMA map
    SKM_TRY(ensure(ctx, ctx->tc_X, sizeof(__half) * (size_t)chunk * (size_t)ctx->tc_h));
    if (ctx->tc_mapX_ptr != ctx->tc_X.p || ctx->tc_mapX_h != ctx->tc_h || ctx->tc_mapX_rows != chunk) {
        SKM_CUDA(tc_make_map(P<__half>(ctx->tc_X), ctx->tc_h, chunk, 128, &ctx->tc_mapX));
        ctx->tc_mapX_ptr = ctx->tc_X.p;
        ctx->tc_mapX_h = ctx->tc_h;
        ctx->tc_mapX_rows = chunk;
    }
    for (int64_t p0 = 0; p0 < sa0.n_list; p0 += chunk) {
        const int32_t n = (int32_t)std::min<int64_t>(chunk, sa0.n_list - p0);
        HeadGemmArgs g{};
        g.hptr = P<int64_t>(ctx->tc_hptr);
        g.hent = P<uint32_t>(ctx->tc_hent);
        g.doc_list = sa0.doc_list;
        g.pos0 = (int32_t)p0;
        g.n = n;
        g.h = ctx->tc_h;
        g.n_cblk = 2 * n_slices;
        g.out = P<__half>(ctx->tc_hs);
        g.ld = ld;
        g.err = P<int32_t>(ctx->counters) + CNT_ERR;
        {
            Timed tm(ctx, ctx->ev_head);
            const int32_t rows = (int32_t)std::min<int64_t>(chunk, ((int64_t)n + 255) / 256 * 256);
            SKM_CUDA(launch_head_rows(g, rows, P<__half>(ctx->tc_X), ctx->st));
            SKM_CUDA(launch_head_gemm(g, ctx->tc_mapX, *map, ctx->st));
        }
        ScoreArgs sa = sa0;
        sa.row_ptr = P<int64_t>(ctx->tc_tptr);
        sa.col = sp ? P<int32_t>(ctx->tc_tcolm) : P<int32_t>(ctx->tc_tcol);
        sa.val = P<float>(ctx->tc_tval);
        sa.pos0 = (int32_t)p0;
        sa.n_list = n;
        sa.n_total = sa0.n_list;
        sa.head = P<__half>(ctx->tc_hs);
        sa.head_ld = ld;
        if (collect) {
            SKM_CUDA(launch_collect(sa, SKM_BF16, ctx->slice, ctx->st, sp));
        } else {
            Timed tm(ctx, ctx->ev_score);
            SKM_CUDA(launch_score(sa, SKM_BF16, ctx->slice, ctx->st, sp));
        }
        ctx->stats.launches_total += 3;
    }
    return SKM_OK;
}

skm_status score_and_decide(skm_ctx *ctx, const DevCsr &dc, const int32_t *list, int32_t n_list,
                            bool pruned, int32_t n_moved, const int32_t *a_old, int32_t *a_new,
                            float *score_out) {
    if (n_list <= 0) return SKM_OK;
    const int32_t k = ctx->cfg.k;
    const int prec = ctx->cfg.precision;
    ScoreArgs sa{};
    sa.row_ptr = dc.row_ptr;
    sa.col = dc.col;
    sa.val = dc.val;
    sa.doc_list = list;
    sa.n_list = n_list;
    sa.ldc = ctx->ldc;
    if (pruned) {
        sa.C = ctx->CM.p;
        sa.ncols = n_moved;
        sa.col_ids = P<int32_t>(ctx->moved);
    } else {
        sa.C = prec == SKM_BF16 ? ctx->C16.p : ctx->C32.p;
        sa.ncols = k;
        sa.col_ids = nullptr;
    }
    sa.part_s = P<float>(ctx->part_s);
    sa.part_j = P<int32_t>(ctx->part_j);
    const int n_slices = (sa.ncols + ctx->slice - 1) / ctx->slice;
    const bool tc = prec == SKM_BF16 && tc_active(ctx);
    if (tc) {
        SKM_TRY(tc_score(ctx, dc, sa, pruned, false));
    } else {
        RareView rv;
        SparseArgs spa{};
        SKM_TRY(ensure_rare(ctx, dc, pruned, sa.ncols, rv));
        const SparseArgs *sp = apply_rare(ctx, rv, sa, spa);
        Timed tm(ctx, ctx->ev_score);
        SKM_CUDA(launch_score(sa, prec, ctx->slice, ctx->st, sp));
    }
    ctx->stats.launches_score++;
    ctx->stats.launches_total++;
    DecideArgs da{};
    da.n_list = n_list;
    da.doc_list = list;
    da.n_slices = n_slices;
    da.n_scored = sa.ncols;
    da.part_s = sa.part_s;
    da.part_j = sa.part_j;
    da.row_ptr = dc.row_ptr;
    da.precision = prec;
    da.head_tc = tc ? 1 : 0;
    da.tau = (float)ctx->cfg.rescore_tau;
    da.rescore = ctx->cfg.rescore;
    da.pruned = pruned ? 1 : 0;
    da.a_old = a_old;
    da.a_new = a_new;
    da.s_state = P<float>(ctx->s_state);
    da.r_state = P<float>(ctx->r_state);
    da.clean = P<uint8_t>(ctx->clean);
    da.score_out = score_out;
    da.counters = P<int32_t>(ctx->counters);
    da.counters64 = P<unsigned long long>(ctx->counters64);
    da.rs_doc = P<int32_t>(ctx->rs_doc);
    da.rs_cand = P<int32_t>(ctx->rs_cand);
    da.refull_doc = P<int32_t>(ctx->refull);
    da.full64_doc = P<int32_t>(ctx->full64);
    da.collect_doc = P<int32_t>(ctx->collect_doc);
    da.collect_thr = P<float>(ctx->collect_thr);
    {
        Timed tm(ctx, ctx->ev_decide);
        SKM_CUDA(launch_decide(da, ctx->st));
    }
    ctx->stats.launches_total++;
    return SKM_OK;
}

// Sum of nonzeros of listed documents (host copy of row_ptr needed): approximated on the
// device side is not needed for correctness; the counters below use the list sizes.
// A bounded wait of the tensor-core scoring kernel gave up (bit 32 of the error counter).
skm_status check_tc_timeout(skm_ctx *ctx) {
    if (ctx->h_counters[CNT_ERR] & 32)
        return fail(ctx, SKM_ERR_TIMEOUT, "a bounded wait of the tensor-core scoring kernel gave up");
    return SKM_OK;
}

skm_status rescore_queues(skm_ctx *ctx, const DevCsr &dc, int32_t *a_new, float *score_out) {
    SKM_TRY(read_counters(ctx));
    SKM_TRY(check_tc_timeout(ctx));
    const int n_rs = ctx->h_counters[CNT_RESCORE];
    const int n_col = ctx->h_counters[CNT_COLLECT];
    RescoreArgs ra{};
    ra.row_ptr = dc.row_ptr;
    ra.col = dc.col;
    ra.val = dc.val;
    ra.C32 = P<float>(ctx->C32);
    ra.ldc = ctx->ldc;
    ra.a_new = a_new;
    ra.score_out = score_out;
    ra.full64_doc = P<int32_t>(ctx->full64);
    ra.full64_count = P<int32_t>(ctx->counters) + CNT_FULL64;
    if (n_rs > 0) {
        // candidate lists of the decision (at most TOPT each)
        ra.count = P<int32_t>(ctx->counters) + CNT_RESCORE;
        ra.rs_doc = P<int32_t>(ctx->rs_doc);
        ra.rs_cand = P<int32_t>(ctx->rs_cand);
        ra.stride = TOPT;
        ra.cand_cnt = nullptr;
        Timed tm(ctx, ctx->ev_decide);
        SKM_CUDA(launch_rescore64(ra, n_rs, ctx->st));
        ctx->stats.launches_total++;
    }
    for (int64_t b0 = 0; b0 < n_col; b0 += kCollectBatch) {
        // more candidates than the list held: collect them all, then rescore those
        const int32_t nb = (int32_t)std::min<int64_t>(kCollectBatch, n_col - b0);
        Timed tm(ctx, ctx->ev_decide);
        SKM_CUDA(cudaMemsetAsync(ctx->cand_cnt.p, 0, sizeof(int32_t) * nb, ctx->st));
        ScoreArgs sa{};
        sa.row_ptr = dc.row_ptr;
        sa.col = dc.col;
        sa.val = dc.val;
        sa.doc_list = P<int32_t>(ctx->collect_doc) + b0;
        sa.n_list = nb;
        sa.C = ctx->cfg.precision == SKM_BF16 ? ctx->C16.p : ctx->C32.p;
        sa.ldc = ctx->ldc;
        sa.ncols = ctx->cfg.k;
        sa.thr = P<float>(ctx->collect_thr) + b0;
        sa.cand_cnt = P<int32_t>(ctx->cand_cnt);
        sa.cand = P<int32_t>(ctx->cand);
        sa.cap = kCollectCap;
        if (ctx->cfg.precision == SKM_BF16 && tc_active(ctx)) {
            // the collect pass recomputes the scoring pass's scores: the same head path
            SKM_TRY(tc_score(ctx, dc, sa, false, true));
        } else {
            RareView rv;
            SparseArgs spa{};
            SKM_TRY(ensure_rare(ctx, dc, false, ctx->cfg.k, rv));
            const SparseArgs *sp = apply_rare(ctx, rv, sa, spa);
            SKM_CUDA(launch_collect(sa, ctx->cfg.precision, ctx->slice, ctx->st, sp));
        }
        ra.count = nullptr;
        ra.n_fixed = nb;
        ra.rs_doc = sa.doc_list;
        ra.rs_cand = sa.cand;
        ra.stride = kCollectCap;
        ra.cand_cnt = sa.cand_cnt;
        SKM_CUDA(launch_rescore64(ra, nb, ctx->st));
        ctx->stats.launches_total += 2;
    }
    int n_f64 = 0;
    if (n_col > 0) {
        SKM_TRY(read_counters(ctx));
        SKM_TRY(check_tc_timeout(ctx));
        n_f64 = ctx->h_counters[CNT_FULL64];
    }
    if (n_f64 > 0) {
        Full64Args fa{};
        fa.count = P<int32_t>(ctx->counters) + CNT_FULL64;
        fa.docs = P<int32_t>(ctx->full64);
        fa.row_ptr = dc.row_ptr;
        fa.col = dc.col;
        fa.val = dc.val;
        fa.C32 = P<float>(ctx->C32);
        fa.ldc = ctx->ldc;
        fa.k = ctx->cfg.k;
        fa.a_new = a_new;
        fa.score_out = score_out;
        Timed tm(ctx, ctx->ev_decide);
        SKM_CUDA(launch_full64(fa, n_f64, ctx->st));
        ctx->stats.launches_total++;
    }
    ctx->stats.docs_rescored += n_rs + n_col - n_f64;
    ctx->stats.docs_rescored_full += n_f64;
    return SKM_OK;
}

// One update step: changed flags, moved list, the two posting passes, objective and shift.
// Returns the number of documents whose assignment changed and |M| through the counters.
// Clears the columns of the clusters recomputed by this update (changed, with members)
// before the write pass. Inside a fit the host knows each column's support (csupport), so
// only its nonzeros are cleared, unless clearing whole columns is cheaper; outside a fit
// (and for unknown supports) whole columns are cleared.
skm_status clear_recomputed(skm_ctx *ctx, const DevCsr &dc, const Postings &pg, const int32_t *a_old, bool sparse) {
    const int32_t k = ctx->cfg.k;
    uint32_t *tiG = ti_current(ctx) ? P<uint32_t>(ctx->ti_G) : nullptr;
    const int32_t tiW = ti_words(k);
    float *C32 = P<float>(ctx->C32);
    __nv_bfloat16 *C16 = ctx->cfg.precision == SKM_BF16 ? P<__nv_bfloat16>(ctx->C16) : nullptr;
    ctx->h_changed.resize(k);
    ctx->h_sizes.resize(k);
    SKM_CUDA(cudaMemcpyAsync(ctx->h_changed.data(), ctx->changed.p, k, cudaMemcpyDeviceToHost, ctx->st));
    SKM_CUDA(cudaMemcpyAsync(ctx->h_sizes.data(), ctx->sizes.p, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, ctx->st));
    SKM_TRY(sync(ctx));
    if ((int32_t)ctx->csupport.size() != k) sparse = false;
    // cost of the member-postings pass (read every posting, scatter a few stores) against
    // clearing whole columns (d rows x recomputed columns x element bytes)
    int64_t n_members = 0, n_rec = 0;
    for (int32_t j = 0; j < k; ++j) {
        if (!ctx->h_changed[j] || ctx->h_sizes[j] == 0) continue;
        ++n_rec;
        if (sparse && ctx->csupport[j] == 0) ++n_members;
    }
    const int64_t elt = C16 ? 6 : 4;
    if (sparse && n_members > 0 && (int64_t)ctx->d * n_members * elt < 2 * 16 * dc.nnz) sparse = false;
    ctx->h_flag.assign(k, 0);
    std::vector<int32_t> seeds;
    ctx->h_list.clear();
    for (int32_t j = 0; j < k; ++j) {
        if (!ctx->h_changed[j] || ctx->h_sizes[j] == 0) continue;
        const uint8_t sup = sparse ? ctx->csupport[j] : 2;
        if (sup == 0) ctx->h_flag[j] = 1;
        else if (sup == 1) seeds.push_back(j);
        else ctx->h_list.push_back(j);
    }
    SKM_TRY(ensure(ctx, ctx->zflag, (size_t)k));
    SKM_TRY(ensure(ctx, ctx->zlist, sizeof(int32_t) * (size_t)k));
    if (n_members > 0 && sparse) {
        SKM_CUDA(cudaMemcpyAsync(ctx->zflag.p, ctx->h_flag.data(), k, cudaMemcpyHostToDevice, ctx->st));
        SKM_CUDA(launch_zero_members(P<int32_t>(ctx->row_idx), P<int32_t>(ctx->pterm), dc.nnz, a_old,
                                     P<uint8_t>(ctx->zflag), C32, C16, ctx->ldc, tiG, tiW, ctx->st));
        ctx->stats.launches_total++;
    }
    if (!seeds.empty()) {
        SKM_CUDA(cudaMemcpyAsync(ctx->zlist.p, seeds.data(), sizeof(int32_t) * seeds.size(), cudaMemcpyHostToDevice,
                                 ctx->st));
        SKM_CUDA(launch_zero_seeds(P<int32_t>(ctx->zlist), (int32_t)seeds.size(), P<int32_t>(ctx->init_ids),
                                   dc.row_ptr, dc.col, C32, C16, ctx->ldc, tiG, tiW, ctx->st));
        ctx->stats.launches_total++;
        SKM_TRY(sync(ctx));   // zlist is reused below
    }
    if (!ctx->h_list.empty()) {
        SKM_CUDA(cudaMemcpyAsync(ctx->zlist.p, ctx->h_list.data(), sizeof(int32_t) * ctx->h_list.size(),
                                 cudaMemcpyHostToDevice, ctx->st));
        SKM_CUDA(launch_zero_cols(P<int32_t>(ctx->zlist), (int32_t)ctx->h_list.size(), ctx->d, C32, C16, ctx->ldc,
                                  tiG, tiW, ctx->st));
        ctx->stats.launches_total++;
    }
    // supports after this update: recomputed -> its new members; a changed cluster left
    // without members keeps its centroid, whose support its members no longer describe
    if ((int32_t)ctx->csupport.size() == k) {
        for (int32_t j = 0; j < k; ++j) {
            if (!ctx->h_changed[j]) continue;
            if (ctx->h_sizes[j] > 0) ctx->csupport[j] = 0;
            else if (ctx->csupport[j] == 0) ctx->csupport[j] = 2;
        }
    }
    SKM_TRY(sync(ctx));   // the host vectors must outlive the copies
    return SKM_OK;
}

skm_status update_step(skm_ctx *ctx, const DevCsr &dc, const Postings &pg, const int32_t *a_new,
                       const int32_t *a_old, int64_t n_docs, bool first, bool converged_check,
                       bool *converged, int iter, bool in_fit) {
    const int32_t k = ctx->cfg.k;
    Timed tm(ctx, ctx->ev_update);
    SKM_CUDA(cudaMemsetAsync(ctx->changed.p, 0, k, ctx->st));
    SKM_CUDA(cudaMemsetAsync(ctx->sizes.p, 0, sizeof(int32_t) * k, ctx->st));
    SKM_CUDA(launch_changed(a_new, a_old, n_docs, first ? 1 : 0, P<uint8_t>(ctx->changed),
                            P<int32_t>(ctx->sizes), k, P<int32_t>(ctx->counters), ctx->st));
    SKM_CUDA(launch_compact_moved(P<uint8_t>(ctx->changed), k, P<int32_t>(ctx->moved),
                                  P<int32_t>(ctx->pos_in_m), P<int32_t>(ctx->counters), ctx->st));
    ctx->stats.launches_total += 2;
    SKM_TRY(read_counters(ctx));
    const int32_t n_changed_docs = ctx->h_counters[CNT_CHANGED];
    const int32_t n_moved = ctx->h_counters[CNT_MOVED];
    *converged = converged_check && !first && n_changed_docs == 0;
    double *obj = P<double>(ctx->obj) + iter;
    double *shf = P<double>(ctx->scal);
    // fixed-point scale of the per-document objective terms (each in [0, 1 + 1e-5])
    int nb = 0;
    while ((int64_t(1) << nb) < n_docs + 1) ++nb;
    const double dot_scale = std::ldexp(1.0, 61 - nb);
    if (!*converged && n_moved > 0) {
        SKM_CUDA(launch_mdoc(a_new, P<int32_t>(ctx->pos_in_m), n_docs, P<int32_t>(ctx->mdoc), ctx->st));
        SKM_CUDA(cudaMemsetAsync(ctx->dot_fx.p, 0, sizeof(unsigned long long) * n_moved, ctx->st));
        SKM_CUDA(launch_doc_obj(dc.row_ptr, dc.col, dc.val, n_docs, a_new, P<int32_t>(ctx->mdoc),
                                P<float>(ctx->C32), ctx->ldc, dot_scale,
                                P<unsigned long long>(ctx->dot_fx), ctx->st));
        UpdateArgs u{};
        u.n_light = pg.n_light;
        u.light_t0 = P<int32_t>(ctx->light_t0);
        u.light_t1 = P<int32_t>(ctx->light_t1);
        u.n_heavy = pg.n_heavy;
        u.heavy_terms = P<int32_t>(ctx->heavy_terms);
        u.n_vh = pg.n_vh;
        u.vh_terms = P<int32_t>(ctx->vh_terms);
        u.vh_sum = P<unsigned long long>(ctx->vh_sum);
        u.n_vch = pg.n_vch;
        u.vch_h = P<int32_t>(ctx->vch_h);
        u.vch_p0 = P<int64_t>(ctx->vch_p0);
        u.vch_p1 = P<int64_t>(ctx->vch_p1);
        u.col_ptr = P<int64_t>(ctx->col_ptr);
        u.row_idx = P<int32_t>(ctx->row_idx);
        u.cval = P<float>(ctx->cval);
        u.pterm = P<int32_t>(ctx->pterm);
        u.mdoc = P<int32_t>(ctx->mdoc);
        u.moved = P<int32_t>(ctx->moved);
        u.n_moved = n_moved;
        u.F = pg.F;
        u.inv_scale = std::ldexp(1.0, -pg.F);
        u.normsq128 = P<unsigned long long>(ctx->normsq128);
        u.sq128 = P<unsigned long long>(ctx->sq128);
        u.inv_norm = P<double>(ctx->inv_norm);
        // the compacted moved matrix serves the next pruned pass; when more than half of the
        // clusters moved and the matrix is large (over 2 GB), the next step scores every
        // document in full instead
        const int64_t cm_bytes = (int64_t)ctx->d * n_moved * (ctx->cfg.precision == SKM_BF16 ? 2 : 4);
        const bool build_cm = in_fit && ctx->cfg.prune != SKM_PRUNE_NONE &&
                              (n_moved <= k / 2 || cm_bytes <= (int64_t(2) << 30));
        u.C32 = P<float>(ctx->C32);
        u.C16 = ctx->cfg.precision == SKM_BF16 ? P<__nv_bfloat16>(ctx->C16) : nullptr;
        u.CM = build_cm ? ctx->CM.p : nullptr;
        u.precision = ctx->cfg.precision;
        u.ldc = ctx->ldc;
        const bool ti_keep = ti_current(ctx);
        if (ti_keep) {
            u.tiG = P<uint32_t>(ctx->ti_G);
            u.tiHist = P<uint32_t>(ctx->ti_hist);
            u.tiW = ti_words(k);
        }
        SKM_CUDA(cudaMemsetAsync(u.normsq128, 0, 2 * sizeof(unsigned long long) * n_moved, ctx->st));
        SKM_CUDA(cudaMemsetAsync(u.sq128, 0, 2 * sizeof(unsigned long long) * n_moved, ctx->st));
        SKM_CUDA(launch_update_vh_sums(u, ctx->st));
        SKM_CUDA(launch_update_norm(u, ctx->st));
        SKM_CUDA(launch_from_u128(u.normsq128, nullptr, n_moved, pg.F, P<double>(ctx->normsq), P<double>(ctx->inv_norm),
                                  nullptr, ctx->st));
        SKM_TRY(clear_recomputed(ctx, dc, pg, a_old, in_fit));
        if (build_cm)
            SKM_CUDA(launch_cm_moved(u.moved, P<int32_t>(ctx->sizes), n_moved, ctx->d, u.C32, u.CM, u.precision,
                                     u.ldc, ctx->st));
        ctx->cm_valid = build_cm;
        if (ti_keep) SKM_CUDA(launch_ti_zero_hist(u.moved, P<int32_t>(ctx->sizes), n_moved, u.tiHist, ctx->st));
        SKM_CUDA(launch_update_write(u, ctx->st));
        SKM_CUDA(launch_from_u128(nullptr, u.sq128, n_moved, pg.F, nullptr, nullptr, P<double>(ctx->newsq), ctx->st));
        ctx->stats.launches_total += 8;
        ctx->cent_epoch++;
        if (ti_keep) ctx->ti_maint_epoch = ctx->cent_epoch;
    }
    // with no moved cluster pos_in_m is -1 everywhere and the objective is sum_j ||S_j||
    SKM_CUDA(launch_finish(P<int32_t>(ctx->pos_in_m), P<int32_t>(ctx->sizes), k,
                           P<unsigned long long>(ctx->dot_fx), 1.0 / dot_scale, P<double>(ctx->normsq),
                           P<double>(ctx->newsq), P<double>(ctx->norm_store), P<double>(ctx->sq_store), obj,
                           shf, ctx->st));
    ctx->stats.launches_total++;
    return SKM_OK;
}

skm_status common_checks(skm_ctx *ctx) {
    if (!ctx) return SKM_ERR_INVALID;
    ctx->err.clear();
    return SKM_OK;
}

}  // namespace

// =====================================================================================
extern "C" {

void skm_config_default(skm_config *cfg, int32_t k) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->k = k;
    cfg->precision = SKM_FP32;
    cfg->prune = SKM_PRUNE_NONE;
    cfg->max_iter = 20;
    cfg->shift_tol = -1.0;
    cfg->rescore = 1;
    cfg->rescore_tau = 0.0;
    cfg->sparse_div = 0;
    cfg->index_levels = 4;
    cfg->index_lambda[0] = 0.1;
    cfg->index_lambda[1] = 0.25;
    cfg->index_lambda[2] = 0.4;
    cfg->index_lambda[3] = 0.6;
    cfg->index_min_changed = 100;
}

skm_status skm_create(const skm_config *cfg, skm_ctx **out) {
    if (!cfg || !out) return SKM_ERR_INVALID;
    *out = nullptr;
    if (cfg->k < 1 || cfg->max_iter < 1 || (cfg->precision != SKM_FP32 && cfg->precision != SKM_BF16) ||
        (cfg->prune != SKM_PRUNE_NONE && cfg->prune != SKM_PRUNE_NCC && cfg->prune != SKM_PRUNE_NCC_INDEX) ||
        cfg->index_max_cands < 0 || cfg->head_terms < -1 ||
        !(cfg->rescore_tau >= 0.0) || (cfg->alloc == nullptr) != (cfg->free == nullptr) || cfg->sparse_div < 0)
        return SKM_ERR_INVALID;
    if (cfg->prune == SKM_PRUNE_NCC_INDEX) {
        if (cfg->index_levels < 1 || cfg->index_levels > TI_MAXL) return SKM_ERR_INVALID;
        for (int l = 0; l < cfg->index_levels; ++l)
            if (!(cfg->index_lambda[l] > 0.0 && cfg->index_lambda[l] <= 1.0) ||
                (l > 0 && !(cfg->index_lambda[l] > cfg->index_lambda[l - 1])))
                return SKM_ERR_INVALID;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return SKM_ERR_CUDA;
    }
    DeviceGuard g(cfg->device);
    skm_ctx *ctx = new skm_ctx();
    ctx->cfg = *cfg;
    ctx->st = (cudaStream_t)cfg->stream;
    ctx->slice = slice_width(cfg->precision, cfg->k);
    ctx->ldc = ((int64_t)cfg->k + ctx->slice - 1) / ctx->slice * ctx->slice;
    ctx->rare_div = cfg->k >= 64 ? cfg->sparse_div : 0;
    if (ensure(ctx, ctx->counters, CNT_N * sizeof(int32_t)) != SKM_OK ||
        ensure(ctx, ctx->counters64, C64_N * sizeof(unsigned long long)) != SKM_OK ||
        cudaMallocHost(&ctx->h_counters64, C64_N * sizeof(unsigned long long)) != cudaSuccess ||
        ensure(ctx, ctx->scal, 8 * sizeof(double)) != SKM_OK ||
        cudaMallocHost(&ctx->h_counters, CNT_N * sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_scal, 8 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        skm_destroy(ctx);
        return SKM_ERR_OOM;
    }
    *out = ctx;
    return SKM_OK;
}

skm_status skm_destroy(skm_ctx *ctx) {
    if (!ctx) return SKM_OK;
    DeviceGuard g(ctx->cfg.device);
    cudaStreamSynchronize(ctx->st);
    Buf *all[] = {&ctx->C32, &ctx->C16, &ctx->CM, &ctx->norm_store, &ctx->d_row_ptr, &ctx->d_col,
                  &ctx->d_val, &ctx->col_ptr, &ctx->row_idx, &ctx->cval, &ctx->pterm, &ctx->tcount,
                  &ctx->light_t0, &ctx->light_t1, &ctx->heavy_terms, &ctx->vh_terms, &ctx->vch_h,
                  &ctx->vch_p0, &ctx->vch_p1, &ctx->vh_sum, &ctx->abuf[0], &ctx->abuf[1], &ctx->s_state, &ctx->r_state,
                  &ctx->clean, &ctx->mdoc, &ctx->order, &ctx->order_hist, &ctx->part_s, &ctx->part_j, &ctx->list_a, &ctx->list_b, &ctx->rs_doc,
                  &ctx->rs_cand, &ctx->refull, &ctx->full64, &ctx->collect_doc, &ctx->collect_thr, &ctx->cand,
                  &ctx->cand_cnt, &ctx->changed, &ctx->sizes, &ctx->moved,
                  &ctx->pos_in_m, &ctx->normsq, &ctx->inv_norm, &ctx->dot_fx, &ctx->newsq,
                  &ctx->rflag, &ctx->rtot, &ctx->rbase, &ctx->rptr_c, &ctx->rent_c, &ctx->rptr_m, &ctx->rent_m,
                  &ctx->colm, &ctx->skipped, &ctx->zflag, &ctx->zlist, &ctx->pp_dist, &ctx->pp_w, &ctx->pp_csum,
                  &ctx->pp_drawn, &ctx->pp_seed, &ctx->pp_ids, &ctx->pp_u, &ctx->ti_G, &ctx->ti_gcnt,
                  &ctx->ti_gptr, &ctx->ti_hist, &ctx->ti_mtab, &ctx->ti_P, &ctx->ti_pbe, &ctx->ti_stats,
                  &ctx->ti_dump, &ctx->ti_scan,
                  &ctx->normsq128, &ctx->sq128, &ctx->sq_store, &ctx->counters, &ctx->counters64, &ctx->scal,
                  &ctx->obj, &ctx->init_ids};
    for (Buf *b : all) release(ctx, *b);
    if (ctx->h_counters) cudaFreeHost(ctx->h_counters);
    if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
    if (ctx->h_counters64) cudaFreeHost(ctx->h_counters64);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    delete ctx;
    return SKM_OK;
}

const char *skm_last_error(const skm_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

skm_status skm_init_kmeanspp(skm_ctx *ctx, const skm_csr *docs, const double *uniforms, int32_t *ids_out) {
    SKM_TRY(common_checks(ctx));
    DeviceGuard g(ctx->cfg.device);
    const int32_t k = ctx->cfg.k;
    if (!uniforms || !ids_out) return fail(ctx, SKM_ERR_INVALID, "uniforms and ids_out are required");
    for (int32_t j = 0; j < k; ++j)
        if (!(uniforms[j] >= 0.0 && uniforms[j] < 1.0))
            return fail(ctx, SKM_ERR_INVALID, "uniforms[%d] = %g is outside [0, 1)", j, uniforms[j]);
    if (docs && docs->n_docs < k)
        return fail(ctx, SKM_ERR_INVALID, "k = %d exceeds n_docs = %lld", k, (long long)docs->n_docs);
    DevCsr dc{};
    SKM_TRY(stage_docs(ctx, docs, dc));
    const int64_t n = dc.n;
    SKM_TRY(ensure(ctx, ctx->pp_dist, sizeof(double) * n));
    SKM_TRY(ensure(ctx, ctx->pp_w, sizeof(unsigned long long) * n));
    SKM_TRY(ensure(ctx, ctx->pp_csum, sizeof(unsigned long long) * kmeanspp_chunks(n)));
    SKM_TRY(ensure(ctx, ctx->pp_drawn, (size_t)n));
    SKM_TRY(ensure(ctx, ctx->pp_seed, sizeof(double) * dc.d));
    SKM_TRY(ensure(ctx, ctx->pp_ids, sizeof(int32_t) * k));
    SKM_TRY(ensure(ctx, ctx->pp_u, sizeof(double) * k));
    SKM_TRY(ensure_doc_bufs(ctx, n));
    // seed 0 = floor(u_0 N)
    int32_t first = (int32_t)std::floor(uniforms[0] * (double)n);
    if (first >= n) first = (int32_t)(n - 1);
    const uint8_t one = 1;
    SKM_CUDA(cudaMemsetAsync(ctx->pp_drawn.p, 0, (size_t)n, ctx->st));
    SKM_CUDA(cudaMemsetAsync(ctx->pp_seed.p, 0, sizeof(double) * dc.d, ctx->st));
    SKM_CUDA(cudaMemcpyAsync(P<uint8_t>(ctx->pp_drawn) + first, &one, 1, cudaMemcpyHostToDevice, ctx->st));
    SKM_CUDA(cudaMemcpyAsync(ctx->pp_ids.p, &first, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->st));
    SKM_CUDA(cudaMemcpyAsync(ctx->pp_u.p, uniforms, sizeof(double) * k, cudaMemcpyHostToDevice, ctx->st));
    SKM_CUDA(launch_order_by_length(dc.row_ptr, n, P<int32_t>(ctx->order_hist), P<int32_t>(ctx->order), ctx->st));
    SKM_CUDA(launch_kmeanspp(n, dc.d, k, P<int32_t>(ctx->order), dc.row_ptr, dc.col, dc.val, P<double>(ctx->pp_u),
                             P<int32_t>(ctx->pp_ids), P<double>(ctx->pp_dist), P<unsigned long long>(ctx->pp_w),
                             P<unsigned long long>(ctx->pp_csum), P<uint8_t>(ctx->pp_drawn), P<double>(ctx->pp_seed),
                             ctx->st));
    std::vector<int32_t> ids(k);
    SKM_CUDA(cudaMemcpyAsync(ids.data(), ctx->pp_ids.p, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, ctx->st));
    SKM_TRY(sync(ctx));
    for (int32_t j = 0; j < k; ++j)
        if (ids[j] < 0 || ids[j] >= n) return fail(ctx, SKM_ERR_CUDA, "k-means++ seed %d out of range", j);
    SKM_CUDA(cudaMemcpyAsync(ids_out, ids.data(), sizeof(int32_t) * k,
                             docs->on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, ctx->st));
    return sync(ctx);
}

skm_status skm_index_candidates(skm_ctx *ctx, const skm_csr *docs, int32_t level, uint32_t *bits) {
    SKM_TRY(common_checks(ctx));
    DeviceGuard g(ctx->cfg.device);
    if (!bits) return fail(ctx, SKM_ERR_INVALID, "bits is NULL");
    if (ctx->d == 0 || !ctx->C32.p) return fail(ctx, SKM_ERR_STATE, "no resident centroids");
    if (ctx->cfg.k > TI_MAX_K) return fail(ctx, SKM_ERR_INVALID, "the threshold index serves k <= %d", TI_MAX_K);
    if (ctx->cfg.index_levels < 1 || ctx->cfg.index_levels > TI_MAXL || level < 0 || level >= ctx->cfg.index_levels)
        return fail(ctx, SKM_ERR_INVALID, "level %d outside [0, %d)", level, ctx->cfg.index_levels);
    for (int l = 0; l < ctx->cfg.index_levels; ++l)
        if (!(ctx->cfg.index_lambda[l] > 0.0 && ctx->cfg.index_lambda[l] <= 1.0))
            return fail(ctx, SKM_ERR_INVALID, "index_lambda[%d] outside (0, 1]", l);
    if (docs && docs->n_terms != ctx->d)
        return fail(ctx, SKM_ERR_INVALID, "n_terms %d differs from the resident vocabulary %d", docs->n_terms, ctx->d);
    DevCsr dc{};
    SKM_TRY(stage_docs(ctx, docs, dc));
    SKM_TRY(build_tindex(ctx));
    const int32_t W = ti_words(ctx->cfg.k);
    const size_t nb = sizeof(uint32_t) * (size_t)dc.n * W;
    SKM_TRY(ensure(ctx, ctx->ti_dump, nb));
    TiQueryArgs qa = ti_args(ctx, dc);
    qa.n_list = dc.n;
    qa.fixed_level = level;
    qa.cand_out = P<uint32_t>(ctx->ti_dump);
    SKM_CUDA(launch_ti_query(qa, ctx->st));
    SKM_CUDA(cudaMemcpyAsync(bits, ctx->ti_dump.p, nb, cudaMemcpyDeviceToHost, ctx->st));
    return sync(ctx);
}

skm_status skm_prepare_assign(skm_ctx *ctx) {
    if (!ctx) return SKM_ERR_INVALID;
    DeviceGuard g(ctx->cfg.device);
    if (ctx->d == 0 || !ctx->C32.p) return SKM_OK;
    SKM_TRY(build_c_index(ctx));
    return sync(ctx);
}

int32_t skm_n_terms(const skm_ctx *ctx) { return ctx ? ctx->d : 0; }

size_t skm_mem_used(const skm_ctx *ctx) { return ctx ? ctx->used : 0; }

skm_status skm_device_code_version(int32_t *out) {
    if (!out) return SKM_ERR_INVALID;
    int v = 0;
    if (score_kernel_version(&v) != cudaSuccess) {
        cudaGetLastError();
        return SKM_ERR_CUDA;
    }
    *out = (int32_t)v;
    return SKM_OK;
}

skm_status skm_get_stats(const skm_ctx *ctx, skm_stats *out) {
    if (!ctx || !out) return SKM_ERR_INVALID;
    *out = ctx->stats;
    return SKM_OK;
}

skm_status skm_fit(skm_ctx *ctx, const skm_csr *docs, const int32_t *init_doc_ids, int32_t *assign_out,
                   double *objective_out, int32_t *iters_out) {
    SKM_TRY(common_checks(ctx));
    DeviceGuard g(ctx->cfg.device);
    const int32_t k = ctx->cfg.k;
    if (!init_doc_ids || !assign_out) return fail(ctx, SKM_ERR_INVALID, "init_doc_ids and assign_out are required");
    if (docs && docs->n_docs < k) return fail(ctx, SKM_ERR_INVALID, "k = %d exceeds n_docs = %lld", k, (long long)docs->n_docs);
    {
        std::vector<char> seen(docs ? (size_t)docs->n_docs : 0, 0);
        for (int32_t j = 0; j < k && docs; ++j) {
            const int32_t id = init_doc_ids[j];
            if (id < 0 || id >= docs->n_docs) return fail(ctx, SKM_ERR_INVALID, "init id %d out of range", id);
            if (seen[id]) return fail(ctx, SKM_ERR_INVALID, "init ids are not distinct (%d)", id);
            seen[id] = 1;
        }
    }
    ctx->stats = skm_stats{};
    ctx->ev_score.clear();
    ctx->ev_decide.clear();
    ctx->ev_update.clear();
    ctx->ev_query.clear();
    ctx->ev_next = 0;
    DevCsr dc{};
    SKM_TRY(stage_docs(ctx, docs, dc));
    const int64_t N = dc.n;
    // the fit lays the centroid matrices out anew: the slice width follows the documents
    ctx->slice = slice_width(ctx->cfg.precision, k, (double)dc.nnz / (double)N);
    ctx->ldc = ((int64_t)k + ctx->slice - 1) / ctx->slice * ctx->slice;
    SKM_TRY(ensure_centroids(ctx, dc.d, true, true));
    SKM_TRY(ensure_cluster_bufs(ctx));
    SKM_TRY(ensure_doc_bufs(ctx, N));
    SKM_TRY(ensure(ctx, ctx->obj, sizeof(double) * ctx->cfg.max_iter));
    SKM_TRY(ensure(ctx, ctx->init_ids, sizeof(int32_t) * k));
    Postings pg;
    SKM_TRY(build_postings(ctx, dc, pg));
    // the head set of the tensor-core scoring path is fixed for the fit (scores stay a pure
    // function of the document and the centroid across its passes)
    SKM_TRY(tc_choose_head(ctx, dc));
    SKM_TRY(tc_split(ctx, dc));
    SKM_CUDA(cudaMemcpyAsync(ctx->init_ids.p, init_doc_ids, sizeof(int32_t) * k, cudaMemcpyHostToDevice, ctx->st));
    SKM_CUDA(launch_init_centroids(dc.row_ptr, dc.col, dc.val, P<int32_t>(ctx->init_ids), k, P<float>(ctx->C32),
                                   ctx->cfg.precision == SKM_BF16 ? P<__nv_bfloat16>(ctx->C16) : nullptr,
                                   ctx->ldc, P<double>(ctx->sq_store), ctx->st));
    ctx->stats.launches_total++;
    ctx->cent_epoch++;
    ctx->csupport.assign(k, 1);   // every column is its seed document
    ctx->cm_valid = false;
    SKM_TRY(reset_skipped(ctx));
    SKM_CUDA(cudaMemsetAsync(ctx->clean.p, 0, N, ctx->st));
    SKM_CUDA(cudaMemsetAsync(ctx->changed.p, 1, k, ctx->st));
    SKM_CUDA(launch_order_by_length(dc.row_ptr, N, P<int32_t>(ctx->order_hist), P<int32_t>(ctx->order), ctx->st));
    ctx->stats.launches_total += 3;

    const bool prune = ctx->cfg.prune != SKM_PRUNE_NONE;
    // the index serves only with a candidate cap configured: in automatic mode (no cap) the
    // dense NCC passes were faster than the index on every workload measured on this GPU
    // (short documents at k = 5000 to 16384 included), so the fit runs them alone
    const bool use_index = ctx->cfg.prune == SKM_PRUNE_NCC_INDEX && k <= TI_MAX_K && ctx->cfg.index_max_cands > 0;
    if (use_index) {
        SKM_TRY(ensure(ctx, ctx->ti_stats, 4 * sizeof(unsigned long long)));
        SKM_CUDA(cudaMemsetAsync(ctx->ti_stats.p, 0, 4 * sizeof(unsigned long long), ctx->st));
    }
    int32_t n_moved_prev = k;
    int32_t it = 0;
    int cur = 0;
    for (int32_t t = 1; t <= ctx->cfg.max_iter; ++t) {
        it = t;
        const bool first = t == 1;
        int32_t *a_old = P<int32_t>(ctx->abuf[cur ^ 1]);
        int32_t *a_new = P<int32_t>(ctx->abuf[cur]);
        SKM_TRY(reset_counters(ctx));
        int32_t n_pruned = 0, n_full = (int32_t)N;
        const int32_t *full_list = P<int32_t>(ctx->order);
        // Sec. 3.2: the threshold index decides the documents whose baseline reaches a
        // threshold when enough centroids changed (Sec. 4.3); the rest go to the dense passes
        const bool index_step = use_index && !first &&
                                (ctx->cfg.index_min_changed < 0 || n_moved_prev > ctx->cfg.index_min_changed);
        if (index_step) {
            SKM_TRY(build_tindex(ctx));
            SKM_CUDA(cudaMemcpyAsync(a_new, a_old, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, ctx->st));
            TiQueryArgs qa = ti_args(ctx, dc);
            qa.n_list = N;
            qa.list = P<int32_t>(ctx->order);
            qa.a_old = a_old;
            qa.changed = P<uint8_t>(ctx->changed);
            qa.ncc = 1;
            qa.prune_fallback = ctx->cm_valid ? 1 : 0;
            qa.a_new = a_new;
            qa.s_state = P<float>(ctx->s_state);
            qa.r_state = P<float>(ctx->r_state);
            qa.clean = P<uint8_t>(ctx->clean);
            qa.counters = P<int32_t>(ctx->counters);
            qa.counters64 = P<unsigned long long>(ctx->counters64);
            qa.pruned_list = P<int32_t>(ctx->list_a);
            qa.full_list = P<int32_t>(ctx->list_b);
            qa.stats = P<unsigned long long>(ctx->ti_stats);
            {
                Timed tm(ctx, ctx->ev_query);
                SKM_CUDA(launch_ti_query(qa, ctx->st));
            }
            ctx->stats.launches_total++;
            SKM_TRY(read_counters(ctx));
            n_pruned = ctx->h_counters[CNT_PRUNED];
            n_full = ctx->h_counters[CNT_FULL];
            full_list = P<int32_t>(ctx->list_b);
        } else if (prune && !first && ctx->cm_valid) {
            // the pruned pass needs the compacted matrix of the last update's moved list
            PartitionArgs pa{};
            pa.n_docs = N;
            pa.order = P<int32_t>(ctx->order);
            pa.prune = 1;
            pa.clean = P<uint8_t>(ctx->clean);
            pa.changed = P<uint8_t>(ctx->changed);
            pa.a_old = a_old;
            pa.row_ptr = dc.row_ptr;
            pa.counters = P<int32_t>(ctx->counters);
            pa.counters64 = P<unsigned long long>(ctx->counters64);
            pa.pruned_list = P<int32_t>(ctx->list_a);
            pa.full_list = P<int32_t>(ctx->list_b);
            SKM_CUDA(launch_partition(pa, ctx->st));
            ctx->stats.launches_total++;
            SKM_TRY(read_counters(ctx));
            n_pruned = ctx->h_counters[CNT_PRUNED];
            n_full = ctx->h_counters[CNT_FULL];
            full_list = P<int32_t>(ctx->list_b);
        }
        // pruned documents keep a_old unless the decision moves them; copy it first
        if (n_pruned > 0 && !index_step) SKM_CUDA(cudaMemcpyAsync(a_new, a_old, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, ctx->st));
        SKM_TRY(score_and_decide(ctx, dc, full_list, n_full, false, k, a_old, a_new, nullptr));
        SKM_TRY(score_and_decide(ctx, dc, P<int32_t>(ctx->list_a), n_pruned, true, n_moved_prev, a_old, a_new, nullptr));
        ctx->stats.docs_full += n_full;
        ctx->stats.docs_pruned += n_pruned;
        ctx->stats.moved_total += n_pruned > 0 ? n_moved_prev : 0;
        ctx->stats.sims += (int64_t)n_full * k + (int64_t)n_pruned * n_moved_prev;
        SKM_TRY(read_counters(ctx));
        const int64_t nnz_pruned = n_pruned > 0 ? (int64_t)ctx->h_counters64[C64_NNZ_PRUNED] : 0;
        const int64_t nnz_full = index_step ? (int64_t)ctx->h_counters64[C64_NNZ_FULL] : dc.nnz - nnz_pruned;
        const int32_t n_refull = ctx->h_counters[CNT_REFULL];
        const int64_t nnz_refull = n_refull > 0 ? (int64_t)ctx->h_counters64[C64_NNZ_REFULL] : 0;
        if (n_refull > 0) {
            SKM_TRY(score_and_decide(ctx, dc, P<int32_t>(ctx->refull), n_refull, false, k, a_old, a_new, nullptr));
            ctx->stats.sims += (int64_t)n_refull * k;
            ctx->stats.docs_full += n_refull;
        }
        // algorithmic work of the scoring passes: one FMA per (nonzero, scored centroid);
        // bytes = CSR entries and per-document state of every scored document, plus each
        // needed centroid element once (rows of present terms x scored columns)
        const int64_t elt = ctx->cfg.precision == SKM_BF16 ? 2 : 4;
        ctx->stats.fmas += nnz_full * k + nnz_pruned * n_moved_prev + nnz_refull * k;
        const int32_t cols_needed = (n_full > 0 || n_refull > 0) ? k : (n_pruned > 0 ? n_moved_prev : 0);
        ctx->stats.bytes += 8 * (nnz_full + nnz_pruned + nnz_refull) + 20 * ((int64_t)n_full + n_pruned + n_refull) +
                            pg.d_eff * cols_needed * elt;
        SKM_TRY(rescore_queues(ctx, dc, a_new, nullptr));
        bool converged = false;
        SKM_TRY(update_step(ctx, dc, pg, a_new, a_old, N, first, true, &converged, t - 1, true));
        n_moved_prev = ctx->h_counters[CNT_MOVED];
        cur ^= 1;
        if (converged) break;
        if (ctx->cfg.shift_tol >= 0.0) {
            SKM_CUDA(cudaMemcpyAsync(ctx->h_scal, ctx->scal.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
            SKM_TRY(sync(ctx));
            if (ctx->h_scal[0] < ctx->cfg.shift_tol) break;
        }
    }
    // the last decided assignment is in abuf[cur ^ 1]
    int32_t *a_fin = P<int32_t>(ctx->abuf[cur ^ 1]);
    SKM_CUDA(cudaMemcpyAsync(assign_out, a_fin, sizeof(int32_t) * N,
                             docs->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->st));
    if (objective_out)
        SKM_CUDA(cudaMemcpyAsync(objective_out, ctx->obj.p, sizeof(double) * it, cudaMemcpyDeviceToHost, ctx->st));
    SKM_TRY(sync(ctx));
    collect_times(ctx);
    ctx->stats.iters = it;
    ctx->stats.head_terms = tc_active(ctx) ? ctx->tc_h : 0;
    ctx->stats.nnz_head = tc_active(ctx) ? ctx->tc_nnz_head : 0;
    if (use_index) {
        unsigned long long h[4];
        SKM_CUDA(cudaMemcpyAsync(h, ctx->ti_stats.p, sizeof h, cudaMemcpyDeviceToHost, ctx->st));
        SKM_TRY(sync(ctx));
        ctx->stats.index_docs = (int64_t)h[0];
        ctx->stats.index_sims = (int64_t)h[1];
        ctx->stats.index_entries = (int64_t)h[2];
        ctx->stats.index_products = (int64_t)h[3];
        ctx->stats.sims += (int64_t)h[1];
    }
    {
        int64_t sk = 0;
        SKM_TRY(read_skipped(ctx, &sk));
        ctx->stats.fmas_exec = ctx->stats.fmas - sk;
    }
    if (iters_out) *iters_out = it;
    return SKM_OK;
}

skm_status skm_assign(skm_ctx *ctx, const skm_csr *docs, int32_t *assign_out, float *score_out) {
    SKM_TRY(common_checks(ctx));
    DeviceGuard g(ctx->cfg.device);
    if (!assign_out) return fail(ctx, SKM_ERR_INVALID, "assign_out is required");
    if (ctx->d == 0 || !ctx->C32.p) return fail(ctx, SKM_ERR_STATE, "no resident centroids");
    if (docs && docs->n_terms != ctx->d)
        return fail(ctx, SKM_ERR_INVALID, "n_terms %d differs from the resident vocabulary %d", docs->n_terms, ctx->d);
    ctx->stats = skm_stats{};
    ctx->ev_next = 0;
    DevCsr dc{};
    SKM_TRY(stage_docs(ctx, docs, dc));
    const int64_t N = dc.n;
    SKM_TRY(ensure_doc_bufs(ctx, N));
    // the head set of the last fit (or of the first assignment on loaded centroids) is kept,
    // so that repeated assignments score every document the same way
    if (ctx->tc_h == 0 || ctx->tc_d != dc.d) {
        if (tc_wanted(ctx)) SKM_TRY(tc_choose_head(ctx, dc));
    }
    SKM_TRY(tc_split(ctx, dc));
    int32_t *a_new = P<int32_t>(ctx->abuf[0]);
    SKM_TRY(reset_counters(ctx));
    SKM_TRY(reset_skipped(ctx));
    // scores go straight to a device output, or through a temporary for a host output
    float *score_dev = nullptr;
    Buf tmp_score;
    if (score_out && !docs->on_device) {
        SKM_TRY(ensure(ctx, tmp_score, sizeof(float) * N));
        score_dev = P<float>(tmp_score);
    } else {
        score_dev = score_out;
    }
    SKM_CUDA(launch_order_by_length(dc.row_ptr, N, P<int32_t>(ctx->order_hist), P<int32_t>(ctx->order), ctx->st));
    ctx->stats.launches_total += 3;
    skm_status s = score_and_decide(ctx, dc, P<int32_t>(ctx->order), (int32_t)N, false, ctx->cfg.k, nullptr, a_new,
                                    score_dev);
    if (s == SKM_OK) s = rescore_queues(ctx, dc, a_new, score_dev);
    if (s == SKM_OK) {
        const cudaMemcpyKind kind = docs->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        cudaError_t e = cudaMemcpyAsync(assign_out, a_new, sizeof(int32_t) * N, kind, ctx->st);
        if (e == cudaSuccess && score_out && !docs->on_device)
            e = cudaMemcpyAsync(score_out, score_dev, sizeof(float) * N, cudaMemcpyDeviceToHost, ctx->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
        if (e != cudaSuccess) s = fail(ctx, SKM_ERR_CUDA, "copy-out failed: %s", cudaGetErrorString(e));
    }
    release(ctx, tmp_score);
    collect_times(ctx);
    ctx->stats.docs_full = N;
    ctx->stats.sims = N * (int64_t)ctx->cfg.k;
    ctx->stats.fmas = dc.nnz * (int64_t)ctx->cfg.k;
    ctx->stats.bytes = 8 * dc.nnz + 20 * N +
                       (int64_t)ctx->d * ctx->cfg.k * (ctx->cfg.precision == SKM_BF16 ? 2 : 4);
    ctx->stats.iters = 1;
    ctx->stats.head_terms = tc_active(ctx) ? ctx->tc_h : 0;
    ctx->stats.nnz_head = tc_active(ctx) ? ctx->tc_nnz_head : 0;
    if (s == SKM_OK) {
        int64_t sk = 0;
        s = read_skipped(ctx, &sk);
        ctx->stats.fmas_exec = ctx->stats.fmas - sk;
    }
    return s;
}

skm_status skm_update(skm_ctx *ctx, const skm_csr *docs, const int32_t *assign, int32_t *n_changed_out) {
    SKM_TRY(common_checks(ctx));
    DeviceGuard g(ctx->cfg.device);
    if (!assign) return fail(ctx, SKM_ERR_INVALID, "assign is required");
    DevCsr dc{};
    SKM_TRY(stage_docs(ctx, docs, dc));
    const int64_t N = dc.n;
    const int32_t k = ctx->cfg.k;
    // assignments: range check on the host copy
    std::vector<int32_t> ha;
    const int32_t *a_dev = nullptr;
    SKM_TRY(ensure_doc_bufs(ctx, N));
    if (docs->on_device) {
        ha.resize(N);
        SKM_CUDA(cudaMemcpyAsync(ha.data(), assign, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, ctx->st));
        SKM_TRY(sync(ctx));
        a_dev = assign;
    } else {
        ha.assign(assign, assign + N);
        SKM_CUDA(cudaMemcpyAsync(ctx->abuf[0].p, assign, sizeof(int32_t) * N, cudaMemcpyHostToDevice, ctx->st));
        a_dev = P<int32_t>(ctx->abuf[0]);
    }
    for (int64_t i = 0; i < N; ++i)
        if (ha[i] < 0 || ha[i] >= k) return fail(ctx, SKM_ERR_INVALID, "assign[%lld] = %d out of range", (long long)i, ha[i]);
    const bool fresh = ctx->d != dc.d;
    SKM_TRY(ensure_centroids(ctx, dc.d, fresh, true));
    SKM_TRY(ensure_cluster_bufs(ctx));
    SKM_TRY(ensure(ctx, ctx->obj, sizeof(double) * std::max(1, ctx->cfg.max_iter)));
    Postings pg;
    SKM_TRY(build_postings(ctx, dc, pg));
    SKM_TRY(reset_counters(ctx));
    bool conv = false;
    ctx->csupport.clear();   // supports are tracked within a fit only
    ctx->cm_valid = false;
    SKM_TRY(update_step(ctx, dc, pg, a_dev, nullptr, N, true, false, &conv, 0, false));
    SKM_TRY(sync(ctx));
    collect_times(ctx);
    if (n_changed_out) *n_changed_out = ctx->h_counters[CNT_MOVED];
    return SKM_OK;
}

skm_status skm_set_centroids(skm_ctx *ctx, int32_t n_terms, const float *centroids, int32_t on_device) {
    SKM_TRY(common_checks(ctx));
    DeviceGuard g(ctx->cfg.device);
    if (n_terms < 1 || !centroids) return fail(ctx, SKM_ERR_INVALID, "n_terms >= 1 and centroids required");
    const int32_t k = ctx->cfg.k;
    SKM_TRY(ensure_centroids(ctx, n_terms, true, false));
    SKM_CUDA(cudaMemcpy2DAsync(ctx->C32.p, sizeof(float) * ctx->ldc, centroids, sizeof(float) * k,
                               sizeof(float) * k, n_terms,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->st));
    // every score is a sum of non-negative products (the decision's all-zero rule and error
    // bounds rest on it): a negative or non-finite entry is rejected and leaves the context
    // without resident centroids
    SKM_TRY(reset_counters(ctx));
    SKM_CUDA(launch_validate_matrix(P<float>(ctx->C32), ctx->ldc, n_terms, k, P<int32_t>(ctx->counters) + CNT_ERR,
                                    ctx->st));
    ctx->stats.launches_total++;
    SKM_TRY(read_counters(ctx));
    if (ctx->h_counters[CNT_ERR]) {
        ctx->d = 0;
        ctx->cent_epoch++;
        ctx->csupport.clear();
        ctx->cm_valid = false;
        return fail(ctx, SKM_ERR_INVALID, "centroids must be finite and non-negative");
    }
    if (ctx->cfg.precision == SKM_BF16) {
        SKM_CUDA(launch_to_bf16(P<float>(ctx->C32), P<__nv_bfloat16>(ctx->C16), (int64_t)n_terms * ctx->ldc, ctx->st));
        ctx->stats.launches_total++;
    }
    ctx->cent_epoch++;
    SKM_CUDA(launch_col_sq(P<float>(ctx->C32), ctx->ldc, n_terms, k, P<double>(ctx->sq_store), ctx->st));
    ctx->csupport.clear();
    ctx->cm_valid = false;
    return sync(ctx);
}

skm_status skm_get_centroids(skm_ctx *ctx, float *out, int32_t on_device) {
    SKM_TRY(common_checks(ctx));
    DeviceGuard g(ctx->cfg.device);
    if (!out) return fail(ctx, SKM_ERR_INVALID, "output is NULL");
    if (ctx->d == 0 || !ctx->C32.p) return fail(ctx, SKM_ERR_STATE, "no resident centroids");
    const int32_t k = ctx->cfg.k;
    SKM_CUDA(cudaMemcpy2DAsync(out, sizeof(float) * k, ctx->C32.p, sizeof(float) * ctx->ldc, sizeof(float) * k,
                               ctx->d, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->st));
    return sync(ctx);
}

}  // extern "C"
