// Serving form: a resident centroid set answers assignment requests by continuous batching
// while clustering jobs run beside it, all under one device-memory budget.
//
//   assign worker  takes every assignment request that is waiting when the GPU becomes free
//                  (up to max_batch_docs documents), concatenates them into one collection,
//                  runs the assignment step on the resident context (its own stream) and
//                  splits the result back; requests that arrive meanwhile join the next batch.
//   job workers    (n_job_slots threads) each take the first waiting clustering job whose
//                  memory estimate fits the free budget, run skm_fit on a context of their own
//                  (own stream, so jobs and assignment batches overlap on the device) and
//                  release the memory. A job that can never fit is rejected at submission.
// Results do not depend on the mix: each document's assignment depends only on the document
// and the resident centroids, and each job is deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "skm.h"
#include "skm_host.h"
#include "skm_internal.cuh"

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum { REQ_ASSIGN = 0, REQ_FIT = 1 };
enum { ST_QUEUED = 0, ST_RUNNING = 1, ST_DONE = 2, ST_REJECTED = 3, ST_FAILED = 4, ST_CANCELLED = 5 };

struct Request {
    uint64_t id = 0;
    int type = REQ_ASSIGN;
    skm_csr docs{};                    // borrowed host arrays (valid until release)
    int32_t k = 0, max_iter = 0;
    std::vector<int32_t> init;
    size_t mem_est = 0;
    std::vector<int32_t> assign;
    std::vector<float> score;
    std::vector<double> objective;
    int32_t iters = 0;
    int state = ST_QUEUED;
    skm_status status = SKM_OK;
    std::string err;
    double t_submit = 0, t_start = 0, t_done = 0;
    int32_t batch_docs = 0;            // size of the batch the request ran in (assign)
};

}  // namespace

struct skm_server {
    skm_server_config cfg{};
    skm_ctx *resident = nullptr;
    std::mutex mu;
    std::condition_variable cv_assign, cv_job, cv_done;
    std::deque<Request *> assign_q, job_q;
    std::unordered_map<uint64_t, Request *> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    size_t jobs_mem = 0;               // estimates of running jobs
    size_t resident_reserve = 0;       // resident centroids + buffers of a largest assign batch
    std::vector<std::thread> threads;
    skm_server_stats stats{};
};

namespace {

// Device memory a clustering job may hold (mirrors the context's allocations, rounded up).
size_t fit_estimate(const skm_csr &d, int32_t k, int precision, int prune) {
    const size_t n = (size_t)d.n_docs, e = (size_t)d.nnz, t = (size_t)d.n_terms;
    const int slice = skm::slice_width(precision, k, (double)e / (double)(n > 0 ? n : 1));
    const size_t ldc = ((size_t)k + slice - 1) / slice * slice;
    const size_t cent = t * ldc * (precision == SKM_BF16 ? (4 + 2 + 2) : (4 + 4));
    const size_t docs = (n + 1) * 8 + e * 8;
    const size_t post = (t + 1) * 12 + e * 12;
    const size_t slices = (ldc + slice - 1) / slice;
    const size_t per_doc = n * (4 * 2 + 4 * 2 + 1 + 4 * 2 + 4 * 6 + 4 * 64 + 4) + n * slices * 4 * 8;
    const size_t per_clus = (size_t)k * 128;
    // sparse-row index of C and of the moved-centroid matrix: a row of either has at most
    // df_t nonzeros, so each holds at most nnz entries; plus the marked column stream
    const size_t esz = precision == SKM_BF16 ? 4 : 8;
    const size_t sparse = e * (4 + 2 * esz) + t * (9 + 2 * (slices + 1) * 4);
    // threshold index (NCC+INDEX): bitmap, per-term offsets and bucket ends, value bins and
    // bounds, and 4 lists of at most nnz entries (a centroid's nonzeros are its members' terms)
    const size_t words = ((size_t)k + 31) / 32;
    const size_t tindex = prune == SKM_PRUNE_NCC_INDEX
                              ? t * (words * 4 + 12 + 4 * 8 * 4) + (size_t)k * 512 * (4 + 4) + 4 * e * 4 +
                                    (size_t)k * 8
                              : 0;
    return (cent + docs + post + per_doc + per_clus + sparse + tindex) * 11 / 10 + (size_t(64) << 20);
}

void assign_worker(skm_server *S) {
    std::vector<int64_t> rp;
    std::vector<int32_t> col, out_a;
    std::vector<float> val, out_s;
    while (true) {
        std::vector<Request *> batch;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_assign.wait(lk, [&] { return S->stop || !S->assign_q.empty(); });
            if (S->stop) return;
            int64_t docs = 0, nnz = 0;
            while (!S->assign_q.empty()) {
                Request *r = S->assign_q.front();
                if (!batch.empty() && (docs + r->docs.n_docs > S->cfg.max_batch_docs ||
                                       nnz + r->docs.nnz > S->cfg.max_batch_nnz))
                    break;
                S->assign_q.pop_front();
                r->state = ST_RUNNING;
                r->t_start = now_ms();
                batch.push_back(r);
                docs += r->docs.n_docs;
                nnz += r->docs.nnz;
            }
        }
        // one collection from the batch (host staging; the library copies it to the device)
        int64_t n = 0, e = 0;
        for (Request *r : batch) { n += r->docs.n_docs; e += r->docs.nnz; }
        rp.resize(n + 1);
        col.resize(e);
        val.resize(e);
        out_a.resize(n);
        out_s.resize(n);
        int64_t dn = 0, de = 0;
        rp[0] = 0;
        for (Request *r : batch) {
            const skm_csr &c = r->docs;
            for (int64_t i = 0; i < c.n_docs; ++i) rp[dn + i + 1] = de + c.row_ptr[i + 1];
            std::memcpy(col.data() + de, c.col_idx, sizeof(int32_t) * c.nnz);
            std::memcpy(val.data() + de, c.values, sizeof(float) * c.nnz);
            dn += c.n_docs;
            de += c.nnz;
        }
        skm_csr all{n, batch[0]->docs.n_terms, e, rp.data(), col.data(), val.data(), 0};
        const skm_status st = skm_assign(S->resident, &all, out_a.data(), out_s.data());
        const std::string err = st == SKM_OK ? "" : skm_last_error(S->resident);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            int64_t off = 0;
            const double t = now_ms();
            for (Request *r : batch) {
                if (st == SKM_OK) {
                    r->assign.assign(out_a.begin() + off, out_a.begin() + off + r->docs.n_docs);
                    r->score.assign(out_s.begin() + off, out_s.begin() + off + r->docs.n_docs);
                    r->state = ST_DONE;
                    S->stats.assign_done++;
                    S->stats.docs_assigned += r->docs.n_docs;
                } else {
                    r->state = ST_FAILED;
                    r->err = err;
                    S->stats.failed++;
                }
                r->status = st;
                r->t_done = t;
                r->batch_docs = (int32_t)n;
                off += r->docs.n_docs;
            }
            S->stats.assign_batches++;
            S->stats.max_batch_docs_seen = std::max<int64_t>(S->stats.max_batch_docs_seen, n);
        }
        S->cv_done.notify_all();
    }
}

void job_worker(skm_server *S) {
    while (true) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_job.wait(lk, [&] {
                if (S->stop) return true;
                const size_t res = S->resident_reserve;
                for (Request *q : S->job_q)
                    if (res + S->jobs_mem + q->mem_est <= S->cfg.mem_budget) return true;
                return false;
            });
            if (S->stop) return;
            const size_t res = S->resident_reserve;
            for (auto it = S->job_q.begin(); it != S->job_q.end(); ++it) {
                if (res + S->jobs_mem + (*it)->mem_est <= S->cfg.mem_budget) {   // first job that fits
                    r = *it;
                    S->job_q.erase(it);
                    break;
                }
            }
            S->jobs_mem += r->mem_est;
            r->state = ST_RUNNING;
            r->t_start = now_ms();
            S->stats.jobs_running++;
            S->stats.peak_jobs_running = std::max(S->stats.peak_jobs_running, S->stats.jobs_running);
        }
        skm_config c;
        skm_config_default(&c, r->k);
        c.precision = S->cfg.job_precision;
        c.prune = S->cfg.job_prune;
        c.max_iter = r->max_iter;
        c.rescore = 1;
        c.rescore_tau = S->cfg.rescore_tau;
        c.mem_budget = r->mem_est;
        c.device = S->cfg.device;
        cudaStream_t st = nullptr;
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(S->cfg.device);
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        c.stream = st;
        skm_ctx *ctx = nullptr;
        skm_status s = skm_create(&c, &ctx);
        std::vector<int32_t> a(r->docs.n_docs);
        std::vector<double> obj(r->max_iter, 0.0);
        int32_t iters = 0;
        std::string err;
        if (s == SKM_OK) {
            s = skm_fit(ctx, &r->docs, r->init.data(), a.data(), obj.data(), &iters);
            if (s != SKM_OK) err = skm_last_error(ctx);
        } else {
            err = "context creation failed";
        }
        skm_destroy(ctx);
        if (st) cudaStreamDestroy(st);
        if (prev >= 0) cudaSetDevice(prev);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->jobs_mem -= r->mem_est;
            S->stats.jobs_running--;
            r->status = s;
            r->t_done = now_ms();
            if (s == SKM_OK) {
                r->assign.swap(a);
                obj.resize(iters);
                r->objective.swap(obj);
                r->iters = iters;
                r->state = ST_DONE;
                S->stats.fit_done++;
                S->stats.docs_clustered += r->docs.n_docs * (int64_t)iters;
            } else {
                r->state = ST_FAILED;
                r->err = err;
                S->stats.failed++;
            }
        }
        S->cv_done.notify_all();
        S->cv_job.notify_all();   // memory was released: waiting jobs may fit now
    }
}

skm_status submit(skm_server *S, Request *r, uint64_t *ticket) {
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    r->t_submit = now_ms();
    S->reqs[r->id] = r;
    *ticket = r->id;
    if (r->type == REQ_FIT) {
        if (S->resident_reserve + r->mem_est > S->cfg.mem_budget) {   // can never fit beside the resident set
            r->state = ST_REJECTED;
            r->status = SKM_ERR_BUDGET;
            r->err = "job memory estimate exceeds the budget left beside the resident centroids";
            r->t_done = r->t_submit;
            S->stats.rejected++;
            S->cv_done.notify_all();
            return SKM_OK;
        }
        S->job_q.push_back(r);
        S->stats.fit_submitted++;
        S->cv_job.notify_one();
    } else {
        S->assign_q.push_back(r);
        S->stats.assign_submitted++;
        S->cv_assign.notify_one();
    }
    return SKM_OK;
}

bool csr_ok(const skm_csr *d) {
    return d && !d->on_device && d->n_docs >= 1 && d->n_terms >= 1 && d->nnz >= d->n_docs && d->row_ptr &&
           d->col_idx && d->values && d->row_ptr[0] == 0 && d->row_ptr[d->n_docs] == d->nnz;
}

}  // namespace

extern "C" {

SKM_API skm_status skm_server_create(const skm_server_config *cfg, skm_ctx *resident, skm_server **out) {
    if (!cfg || !resident || !out || cfg->n_job_slots < 0 || cfg->max_batch_docs < 1 ||
        cfg->max_batch_nnz < cfg->max_batch_docs || cfg->mem_budget == 0 ||
        (cfg->job_precision != SKM_FP32 && cfg->job_precision != SKM_BF16) || !(cfg->rescore_tau >= 0.0))
        return SKM_ERR_INVALID;
    if (skm_n_terms(resident) < 1) return SKM_ERR_STATE;
    if (skm_prepare_assign(resident) != SKM_OK) return SKM_ERR_CUDA;
    // memory kept for the resident context: what it holds now (centroids and their
    // sparse-row index) plus the per-document, staging and marked-column buffers of a
    // largest batch (they grow on demand up to this size)
    const size_t nd = (size_t)cfg->max_batch_docs, ne = (size_t)cfg->max_batch_nnz;
    const size_t reserve = skm_mem_used(resident) + ((nd + 1) * 8 + ne * 12 + nd * (48 + 4 * 64 + 32 * 32)) * 11 / 10 +
                           (size_t(64) << 20);
    if (reserve > cfg->mem_budget) return SKM_ERR_BUDGET;
    skm_server *S = new skm_server();
    S->cfg = *cfg;
    S->resident = resident;
    S->resident_reserve = reserve;
    S->threads.emplace_back(assign_worker, S);
    for (int i = 0; i < cfg->n_job_slots; ++i) S->threads.emplace_back(job_worker, S);
    *out = S;
    return SKM_OK;
}

SKM_API skm_status skm_server_submit_assign(skm_server *S, const skm_csr *docs, uint64_t *ticket) {
    if (!S || !ticket || !csr_ok(docs)) return SKM_ERR_INVALID;
    if (docs->n_terms != skm_n_terms(S->resident)) return SKM_ERR_INVALID;
    if (docs->n_docs > S->cfg.max_batch_docs) return SKM_ERR_INVALID;
    Request *r = new Request();
    r->type = REQ_ASSIGN;
    r->docs = *docs;
    return submit(S, r, ticket);
}

SKM_API skm_status skm_server_submit_fit(skm_server *S, const skm_csr *docs, int32_t k, const int32_t *init_doc_ids,
                                         int32_t max_iter, uint64_t *ticket) {
    if (!S || !ticket || !csr_ok(docs) || k < 1 || k > docs->n_docs || !init_doc_ids || max_iter < 1)
        return SKM_ERR_INVALID;
    Request *r = new Request();
    r->type = REQ_FIT;
    r->docs = *docs;
    r->k = k;
    r->max_iter = max_iter;
    r->init.assign(init_doc_ids, init_doc_ids + k);
    r->mem_est = fit_estimate(*docs, k, S->cfg.job_precision, S->cfg.job_prune);
    return submit(S, r, ticket);
}

SKM_API skm_status skm_server_wait(skm_server *S, uint64_t ticket, double timeout_ms, skm_server_result *res) {
    if (!S || !res) return SKM_ERR_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return SKM_ERR_INVALID;
    Request *r = it->second;
    auto done = [&] { return r->state >= ST_DONE; };
    if (timeout_ms < 0) S->cv_done.wait(lk, done);
    else S->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), done);
    std::memset(res, 0, sizeof(*res));
    res->state = r->state;
    res->status = r->status;
    res->n_docs = r->docs.n_docs;
    res->assign = r->assign.empty() ? nullptr : r->assign.data();
    res->score = r->score.empty() ? nullptr : r->score.data();
    res->objective = r->objective.empty() ? nullptr : r->objective.data();
    res->iters = r->iters;
    res->latency_ms = r->state >= ST_DONE ? r->t_done - r->t_submit : -1.0;
    res->queue_ms = r->t_start > 0 ? r->t_start - r->t_submit : -1.0;
    res->batch_docs = r->batch_docs;
    std::snprintf(res->message, sizeof res->message, "%s", r->err.c_str());
    return r->state >= ST_DONE ? SKM_OK : SKM_ERR_TIMEOUT;
}

SKM_API skm_status skm_server_release(skm_server *S, uint64_t ticket) {
    if (!S) return SKM_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return SKM_ERR_INVALID;
    if (it->second->state < ST_DONE) return SKM_ERR_STATE;
    delete it->second;
    S->reqs.erase(it);
    return SKM_OK;
}

SKM_API skm_status skm_server_get_stats(skm_server *S, skm_server_stats *out) {
    if (!S || !out) return SKM_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    out->assign_queued = (int64_t)S->assign_q.size();
    out->fit_queued = (int64_t)S->job_q.size();
    out->jobs_mem = S->jobs_mem;
    out->resident_mem = S->resident_reserve;
    return SKM_OK;
}

SKM_API skm_status skm_server_destroy(skm_server *S) {
    if (!S) return SKM_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (Request *r : S->assign_q) r->state = ST_CANCELLED;
        for (Request *r : S->job_q) r->state = ST_CANCELLED;
        S->assign_q.clear();
        S->job_q.clear();
    }
    S->cv_assign.notify_all();
    S->cv_job.notify_all();
    S->cv_done.notify_all();
    for (auto &t : S->threads) t.join();   // running work finishes first
    for (auto &kv : S->reqs) delete kv.second;
    delete S;
    return SKM_OK;
}

}  // extern "C"
