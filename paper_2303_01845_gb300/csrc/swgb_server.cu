// swgb_server.cu -- a query server over a resident reference set: requests
// (batches of query sequences) are admitted by device memory into worker
// slots, and each admitted batch runs the whole search on its slot's own
// context and stream -- shared-k-mer candidates from the resident index, the
// learned filter, exact alignment, identity and pass / fail -- so that the
// batches of different slots overlap on the GPU while new requests wait for
// a slot and for memory.
//
// The paper's system is a batch job (Sec. "Protein similarity search
// pipeline"); serving is this library's: the resident index plays the role
// of the paper's distributed sequence-by-k-mer matrix of the references,
// and admission by memory follows the paper's blocked formation of the
// overlap matrix, which bounds the memory of each block (Sec. "Blocked 2D
// Sparse SUMMA").
//
// Host-only code on top of the public C ABI; every device step is a
// libswgb call.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "swgb.h"

#define SWGB_EXPORT extern "C" __attribute__((visibility("default")))

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket = 0;
    std::vector<uint8_t> res;       // codes
    std::vector<int64_t> off;       // n + 1, from 0
    int64_t n = 0;
    int64_t reserve = 0;            // bytes held while in flight
    Clock::time_point submitted, admitted, finished;
    bool done = false;
    int status = SWGB_OK;
    std::string error;
    // results, pairs (query index within the request, reference index)
    std::vector<int32_t> pairs;
    std::vector<int32_t> counts;
    std::vector<swgb_record> records;
    std::vector<swgb_identity_record> ident;
    int64_t candidates = 0;
    int64_t batch_id = -1;
    int32_t slot = -1;
    double stage_ms[SWGB_SERVER_STAGES] = {};   // of the batch it ran in
};

// Device buffers of a slot, grown on demand.
template <class T>
struct DevBuf {
    T* p = nullptr;
    int64_t cap = 0;
    cudaError_t need(int64_t n) {
        if (n <= cap && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        const int64_t c = std::max<int64_t>(n, cap * 3 / 2 + 1);
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), sizeof(T) * (size_t)c);
        if (e == cudaSuccess) cap = c;
        return e;
    }
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

}  // namespace

struct swgb_server {
    int device = 0;
    const swgb_index* index = nullptr;
    const swgb_seqset* refs = nullptr;
    std::vector<int8_t> matrix;
    swgb_params params{};
    swgb_server_config cfg{};
    std::vector<float> mlp_params;   // empty: no filter
    bool use_filter = false;

    std::mutex mu;
    std::condition_variable cv_work;   // workers: a request arrived or memory freed
    std::condition_variable cv_done;   // waiters: a request finished
    std::deque<std::shared_ptr<Request>> pending;
    std::map<int64_t, std::shared_ptr<Request>> requests;
    int64_t next_ticket = 1;
    int64_t next_batch = 1;
    int64_t inflight_bytes = 0;
    int32_t inflight_batches = 0;
    int32_t max_overlap = 0;         // most batches seen in flight at once
    bool stopping = false;
    std::vector<std::thread> workers;
    std::string err;
};

namespace {

// Bytes a request holds on the device while in flight: its residues' k-mer
// tables and the candidates it is expected to produce (per query:
// cfg.candidates_per_query of pairs, features, logits, records, identity).
int64_t reservation(const swgb_server* s, int64_t residues, int64_t n) {
    const int64_t per_candidate = 8 + 4 + 128 + 4 + 8 + 8 + 20 + 12;
    return residues * 24 + n * (int64_t)s->cfg.candidates_per_query * per_candidate;
}

void finish(swgb_server* s, std::vector<std::shared_ptr<Request>>& batch, int status,
            const std::string& msg) {
    std::lock_guard<std::mutex> lk(s->mu);
    const auto now = Clock::now();
    for (auto& r : batch) {
        r->status = status;
        if (status != SWGB_OK) r->error = msg;
        r->finished = now;
        r->done = true;
        s->inflight_bytes -= r->reserve;
    }
    s->inflight_batches -= 1;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

// Takes the longest FIFO prefix of the pending requests that fits one batch
// and the memory budget (blocks while none fits).  Returns false to stop.
bool admit(swgb_server* s, std::vector<std::shared_ptr<Request>>& batch, int64_t* batch_id) {
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        if (s->stopping) return false;
        if (!s->pending.empty()) {
            int64_t residues = 0, bytes = 0, queries = 0;
            for (auto& r : s->pending) {
                const int64_t nr = residues + (int64_t)r->res.size();
                const int64_t nb = bytes + r->reserve;
                if (!batch.empty() && (nr > s->cfg.max_batch_residues ||
                                       queries + r->n > s->cfg.max_batch_queries))
                    break;
                if (s->inflight_bytes + nb > s->cfg.max_inflight_bytes) break;
                batch.push_back(r);
                residues = nr;
                bytes = nb;
                queries += r->n;
            }
            if (!batch.empty()) {
                const auto now = Clock::now();
                for (size_t k = 0; k < batch.size(); ++k) {
                    s->pending.pop_front();
                    batch[k]->admitted = now;
                }
                s->inflight_bytes += bytes;
                s->inflight_batches += 1;
                s->max_overlap = std::max(s->max_overlap, s->inflight_batches);
                *batch_id = s->next_batch++;
                // requests left over: wake another idle worker for them
                if (!s->pending.empty()) s->cv_work.notify_one();
                return true;
            }
        }
        s->cv_work.wait(lk);
    }
}

struct Slot {
    swgb_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    swgb_seqset* queries = nullptr;
    swgb_mlp* mlp = nullptr;
    DevBuf<int32_t> cand, counts, kept;
    DevBuf<int64_t> kept_index;
    DevBuf<float> feats, logits;
    DevBuf<swgb_record> rec;
    DevBuf<swgb_identity_record> ident;
};

#define SCK(call)                                                      \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return fail_batch(std::string(#call) + ": " + cudaGetErrorString(e_), SWGB_ECUDA); \
    } while (0)

void worker(swgb_server* s, int slot_id) {
    cudaSetDevice(s->device);
    Slot sl;
    std::string setup_err;
    if (swgb_create(s->device, &sl.ctx) != SWGB_OK) setup_err = "swgb_create failed";
    if (setup_err.empty() && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess)
        setup_err = "cudaStreamCreate failed";
    if (setup_err.empty() && s->use_filter &&
        swgb_mlp_create(sl.ctx, s->mlp_params.data(), &sl.mlp) != SWGB_OK)
        setup_err = std::string("swgb_mlp_create: ") + swgb_last_error(sl.ctx);
    for (;;) {
        std::vector<std::shared_ptr<Request>> batch;
        int64_t batch_id = 0;
        if (!admit(s, batch, &batch_id)) break;
        for (auto& r : batch) {
            r->batch_id = batch_id;
            r->slot = slot_id;
        }
        auto fail_batch = [&](const std::string& msg, int code) {
            finish(s, batch, code, msg);
            return 0;
        };
        if (!setup_err.empty()) {
            fail_batch(setup_err, SWGB_ECUDA);
            continue;
        }
        double stage[SWGB_SERVER_STAGES] = {};
        auto t_mark = Clock::now();
        auto lap = [&](int k) {
            const auto now = Clock::now();
            stage[k] += std::chrono::duration<double, std::milli>(now - t_mark).count();
            t_mark = now;
        };
        auto run = [&]() -> int {
            // the batch's queries, concatenated
            std::vector<uint8_t> res;
            std::vector<int64_t> off(1, 0);
            std::vector<int64_t> first;   // first query index of each request
            for (auto& r : batch) {
                first.push_back((int64_t)off.size() - 1);
                const int64_t base = (int64_t)res.size();
                res.insert(res.end(), r->res.begin(), r->res.end());
                for (int64_t q = 1; q <= r->n; ++q) off.push_back(base + r->off[q]);
            }
            const int64_t nq = (int64_t)off.size() - 1;
            int rc = sl.queries ? swgb_seqset_load(sl.queries, res.data(), off.data(), nq, 0, sl.stream)
                                : swgb_seqset_create(sl.ctx, res.data(), off.data(), nq, 0, sl.stream,
                                                     &sl.queries);
            if (rc) return fail_batch(std::string("queries: ") + swgb_last_error(sl.ctx), rc);
            lap(0);
            // candidates from the resident index
            int64_t found = 0;
            SCK(sl.cand.need(2 * std::max<int64_t>(sl.cand.cap / 2, 1024)));
            SCK(sl.counts.need(sl.cand.cap / 2));
            int64_t cap = std::min(sl.cand.cap / 2, sl.counts.cap);
            rc = swgb_index_query(sl.ctx, s->index, sl.queries, s->cfg.min_shared, sl.cand.p,
                                  sl.counts.p, cap, &found, sl.stream);
            if (rc) return fail_batch(std::string("index_query: ") + swgb_last_error(sl.ctx), rc);
            if (found > cap) {
                SCK(sl.cand.need(2 * found));
                SCK(sl.counts.need(found));
                cap = found;
                rc = swgb_index_query(sl.ctx, s->index, sl.queries, s->cfg.min_shared, sl.cand.p,
                                      sl.counts.p, cap, &found, sl.stream);
                if (rc) return fail_batch(std::string("index_query: ") + swgb_last_error(sl.ctx), rc);
            }
            lap(1);
            const int32_t* align_pairs = sl.cand.p;
            int64_t n_align = found;
            if (sl.mlp && found > 0) {
                SCK(sl.feats.need(found * SWGB_FEATURES));
                SCK(sl.logits.need(found));
                SCK(sl.kept.need(2 * found));
                SCK(sl.kept_index.need(found));
                rc = swgb_index_features(sl.ctx, s->index, sl.queries, sl.cand.p, found, sl.feats.p,
                                         sl.stream);
                if (!rc) rc = swgb_mlp_forward(sl.mlp, sl.feats.p, found, sl.logits.p, sl.stream);
                if (!rc) rc = swgb_select_pairs(sl.ctx, sl.cand.p, sl.logits.p, found, s->cfg.threshold,
                                                sl.kept.p, sl.kept_index.p, &n_align, sl.stream);
                if (rc) return fail_batch(std::string("filter: ") + swgb_last_error(sl.ctx), rc);
                align_pairs = sl.kept.p;
            }
            lap(2);
            SCK(sl.rec.need(std::max<int64_t>(n_align, 1)));
            SCK(sl.ident.need(std::max<int64_t>(n_align, 1)));
            if (n_align > 0) {
                rc = swgb_align(sl.ctx, sl.queries, s->refs, align_pairs, n_align, &s->params, sl.rec.p,
                                sl.stream);
                if (!rc) rc = swgb_identity(sl.ctx, sl.queries, s->refs, align_pairs, sl.rec.p, n_align,
                                            &s->params, &s->cfg.identity, sl.ident.p, sl.stream);
                if (!rc) rc = swgb_sync(sl.ctx, sl.stream);
                if (rc) return fail_batch(std::string("align: ") + swgb_last_error(sl.ctx), rc);
            }
            lap(3);
            // results back, split per request (pairs are ordered by query)
            std::vector<int32_t> hp((size_t)(2 * n_align)), hc((size_t)found);
            std::vector<swgb_record> hr((size_t)n_align);
            std::vector<swgb_identity_record> hi((size_t)n_align);
            std::vector<int64_t> hk;
            if (n_align > 0) {
                SCK(cudaMemcpyAsync(hp.data(), align_pairs, sizeof(int32_t) * 2 * n_align,
                                    cudaMemcpyDeviceToHost, sl.stream));
                SCK(cudaMemcpyAsync(hr.data(), sl.rec.p, sizeof(swgb_record) * n_align,
                                    cudaMemcpyDeviceToHost, sl.stream));
                SCK(cudaMemcpyAsync(hi.data(), sl.ident.p, sizeof(swgb_identity_record) * n_align,
                                    cudaMemcpyDeviceToHost, sl.stream));
                if (sl.mlp) {
                    hk.resize((size_t)n_align);
                    SCK(cudaMemcpyAsync(hk.data(), sl.kept_index.p, sizeof(int64_t) * n_align,
                                        cudaMemcpyDeviceToHost, sl.stream));
                }
            }
            if (found > 0)
                SCK(cudaMemcpyAsync(hc.data(), sl.counts.p, sizeof(int32_t) * found,
                                    cudaMemcpyDeviceToHost, sl.stream));
            SCK(cudaStreamSynchronize(sl.stream));
            // candidates per query of the batch, before the filter
            std::vector<int64_t> per_query_found((size_t)nq + 1, 0);
            if (found > 0) {
                std::vector<int32_t> all((size_t)(2 * found));
                SCK(cudaMemcpyAsync(all.data(), sl.cand.p, sizeof(int32_t) * 2 * found,
                                    cudaMemcpyDeviceToHost, sl.stream));
                SCK(cudaStreamSynchronize(sl.stream));
                for (int64_t c = 0; c < found; ++c) per_query_found[(size_t)all[2 * c]] += 1;
            }
            size_t p = 0;
            for (size_t b = 0; b < batch.size(); ++b) {
                Request& r = *batch[b];
                const int64_t q0 = first[b], q1 = q0 + r.n;
                r.candidates = 0;
                for (int64_t q = q0; q < q1; ++q) r.candidates += per_query_found[(size_t)q];
                while (p < (size_t)n_align && hp[2 * p] < q1) {
                    r.pairs.push_back(hp[2 * p] - (int32_t)q0);
                    r.pairs.push_back(hp[2 * p + 1]);
                    r.counts.push_back(hc[(size_t)(sl.mlp ? hk[p] : (int64_t)p)]);
                    r.records.push_back(hr[p]);
                    r.ident.push_back(hi[p]);
                    ++p;
                }
            }
            lap(4);
            for (auto& r : batch)
                for (int k = 0; k < SWGB_SERVER_STAGES; ++k) r->stage_ms[k] = stage[k];
            finish(s, batch, SWGB_OK, "");
            return 0;
        };
        run();
    }
    if (sl.mlp) swgb_mlp_destroy(sl.mlp);
    if (sl.queries) swgb_seqset_destroy(sl.queries);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ctx) swgb_destroy(sl.ctx);
}

}  // namespace

SWGB_EXPORT void swgb_server_default_config(swgb_server_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->slots = 3;
    cfg->max_batch_queries = 4096;
    cfg->max_batch_residues = 1 << 20;
    cfg->max_inflight_bytes = (int64_t)4 << 30;
    cfg->candidates_per_query = 256;
    cfg->min_shared = 2;
    cfg->threshold = 0.0f;
    cfg->identity = swgb_thresholds{3, 10, 7, 10};
}

SWGB_EXPORT int swgb_server_create(int device, const swgb_seqset* refs, const swgb_index* index,
                                   const float* mlp_params, const swgb_params* params,
                                   const swgb_server_config* cfg, swgb_server** out) {
    if (!out || !refs || !index || !params || !params->matrix || !cfg) return SWGB_EINVAL;
    *out = nullptr;
    if (cfg->slots < 1 || cfg->slots > 64 || cfg->max_batch_queries < 1 ||
        cfg->max_batch_residues < 1 || cfg->max_inflight_bytes < 1 || cfg->min_shared < 1 ||
        cfg->candidates_per_query < 0)
        return SWGB_EINVAL;
    swgb_server* s = new (std::nothrow) swgb_server();
    if (!s) return SWGB_ENOMEM;
    s->device = device;
    s->index = index;
    s->refs = refs;
    s->matrix.assign(params->matrix, params->matrix + SWGB_ALPHABET_SIZE * SWGB_ALPHABET_SIZE);
    s->params = *params;
    s->params.matrix = s->matrix.data();
    s->params.flags &= ~SWGB_TIMING;
    s->cfg = *cfg;
    if (mlp_params) {
        s->mlp_params.assign(mlp_params, mlp_params + SWGB_MLP_PARAMS);
        s->use_filter = true;
    }
    for (int k = 0; k < cfg->slots; ++k) s->workers.emplace_back(worker, s, k);
    *out = s;
    return SWGB_OK;
}

SWGB_EXPORT void swgb_server_destroy(swgb_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
}

SWGB_EXPORT int swgb_server_submit(swgb_server* s, const uint8_t* codes, const int64_t* offsets,
                                   int64_t n_queries, int64_t* ticket) {
    if (!s || !ticket || n_queries < 1 || !offsets) return SWGB_EINVAL;
    *ticket = 0;
    auto r = std::make_shared<Request>();
    r->n = n_queries;
    const int64_t base = offsets[0];
    for (int64_t q = 0; q <= n_queries; ++q) {
        if (q > 0 && offsets[q] < offsets[q - 1]) return SWGB_ERANGE;
        r->off.push_back(offsets[q] - base);
    }
    const int64_t total = r->off.back();
    if (total > 0 && !codes) return SWGB_EINVAL;
    r->res.assign(codes + base, codes + base + total);
    for (uint8_t c : r->res)
        if (c >= SWGB_ALPHABET_SIZE) return SWGB_EBADRES;
    r->reserve = reservation(s, total, n_queries);
    if (total > s->cfg.max_batch_residues || n_queries > s->cfg.max_batch_queries ||
        r->reserve > s->cfg.max_inflight_bytes)
        return SWGB_ETOOBIG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) return SWGB_EINVAL;
        r->ticket = s->next_ticket++;
        r->submitted = Clock::now();
        s->pending.push_back(r);
        s->requests[r->ticket] = r;
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return SWGB_OK;
}

SWGB_EXPORT int swgb_server_wait(swgb_server* s, int64_t ticket, int64_t timeout_ms,
                                 swgb_server_result* out) {
    if (!s || !out) return SWGB_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->requests.find(ticket);
    if (it == s->requests.end()) return SWGB_EINVAL;
    std::shared_ptr<Request> r = it->second;
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (!r->done) {
        if (timeout_ms < 0) {
            s->cv_done.wait(lk);
        } else if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done) {
            return SWGB_ETIMEDOUT;
        }
    }
    std::memset(out, 0, sizeof(*out));
    out->status = r->status;
    out->n_pairs = (int64_t)r->records.size();
    out->n_candidates = r->candidates;
    out->pairs = r->pairs.data();
    out->counts = r->counts.data();
    out->records = r->records.data();
    out->identity = r->ident.data();
    out->queue_ms = std::chrono::duration<double, std::milli>(r->admitted - r->submitted).count();
    out->latency_ms = std::chrono::duration<double, std::milli>(r->finished - r->submitted).count();
    out->batch_id = r->batch_id;
    out->slot = r->slot;
    out->error = r->error.c_str();
    for (int k = 0; k < SWGB_SERVER_STAGES; ++k) out->stage_ms[k] = r->stage_ms[k];
    return SWGB_OK;
}

SWGB_EXPORT int swgb_server_release(swgb_server* s, int64_t ticket) {
    if (!s) return SWGB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->requests.find(ticket);
    if (it == s->requests.end() || !it->second->done) return SWGB_EINVAL;
    s->requests.erase(it);
    return SWGB_OK;
}

SWGB_EXPORT int swgb_server_stats(swgb_server* s, int32_t* max_overlap, int64_t* pending,
                                  int64_t* inflight_bytes) {
    if (!s) return SWGB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (max_overlap) *max_overlap = s->max_overlap;
    if (pending) *pending = (int64_t)s->pending.size();
    if (inflight_bytes) *inflight_bytes = s->inflight_bytes;
    return SWGB_OK;
}
