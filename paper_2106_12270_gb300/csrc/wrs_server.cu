// wrs_server.cu - a continuous-batching request loop over resident tables.
//
// Requests (build a table, draw samples from a resident table, release a
// table) are queued by any thread and served by one worker thread:
//   * admission: a build is admitted only while the HBM budget has room for
//     its rows (resident until released) and its transient scratch; builds
//     keep their arrival order, samples and releases are never held back by
//     a waiting build;
//   * each step gathers every admissible request that has arrived, builds all
//     of its small tables with one batched-build launch (one CTA per table)
//     and each large table (kLargeBuild items or more) with the multi-CTA
//     single-table pipeline, and draws all of its samples with one
//     request-sampling launch, on two streams; a sample of a table built in
//     an earlier step that is still running waits for that table's event on
//     the GPU, not on the host;
//   * up to max_inflight steps are on the GPU at once, and requests that
//     arrive meanwhile go into the next step, so new work overlaps running
//     work (continuous batching, not a queue drained one batch at a time).
// A request's result does not depend on what it is batched with: tables are
// built by the same exact arithmetic as a single build, and request samples
// use the counters of wrs_sample_rows (seed, stream_lo, WRS_TAG_NAIVE).
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wrs_internal.cuh"

namespace wrs {


cudaError_t launch_sample_requests(const SampleReq *, const uint32_t *, uint32_t, uint32_t,
                                   cudaStream_t);
cudaError_t launch_total(const float *, uint64_t, unsigned char *, const Layout &, cudaStream_t);
cudaError_t launch_partition(const float *, uint64_t, unsigned char *, const Layout &,
                             cudaStream_t);
cudaError_t launch_split(uint64_t, unsigned char *, const Layout &, uint32_t, uint32_t,
                         cudaStream_t);
cudaError_t launch_pack(uint64_t, wrs_row *, unsigned char *, const Layout &, uint32_t,
                        cudaStream_t);
cudaError_t launch_info(unsigned char *, const Layout &, wrs_build_info *, cudaStream_t);
int cuda_status(cudaError_t e);

// A table this large is built by the multi-CTA single-table pipeline: one CTA
// of the batched kernel would sweep it alone for milliseconds.
constexpr uint64_t kLargeBuild = 1ull << 17;
constexpr uint32_t kLargeSection = 1024;
constexpr uint64_t kMaxServerItems = (1ull << 31) - 1;
constexpr uint64_t kReqChunkH = 1u << 16;         // samples per CTA of the request sampler
constexpr uint32_t kMaxReqPerStep = 8192;

static double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum Kind { K_BUILD, K_SAMPLE, K_RELEASE };

struct Request {
    uint64_t id = 0;
    Kind kind = K_BUILD;
    const float *w = nullptr;
    uint64_t n = 0;
    int w_dev = 0;
    uint64_t table = 0;
    uint64_t count = 0, seed = 0;
    uint32_t slo = 0;
    uint32_t *out = nullptr;
    int out_dev = 0;
    double t_submit = 0, t_done = 0;
    int status = WRS_OK;
    bool done = false;
    // sample staging (host outputs)
    uint64_t stage_off = 0;
};

struct TableRec {
    wrs_row *rows = nullptr;
    uint64_t n = 0, bytes = 0;
    int status = WRS_OK;
    bool built = false;      // its build step has retired
    bool gone = false;       // released or failed
    cudaEvent_t ready = nullptr;
    double W = 0;
    uint64_t nl = 0, nh = 0;
};

struct Slot {   // pinned staging reused by one in-flight step
    unsigned char *pin = nullptr;
    uint64_t pin_bytes = 0;
    uint32_t *pin_out = nullptr;
    uint64_t pin_out_bytes = 0;
    bool busy = false;
};

struct Step {
    cudaEvent_t done = nullptr, built = nullptr;
    std::vector<Request *> reqs;
    std::vector<uint64_t> tables;   // built in this step, in summary order
    std::vector<uint64_t> ltables;  // large tables built in this step, in linfo order
    std::vector<void *> lscratch;   // their weights + workspaces
    wrs_build_info *linfo = nullptr;    // pinned
    void *scratch = nullptr;
    uint64_t scratch_bytes = 0;
    int slot = -1;
    wrs_table_summary *summ = nullptr;   // pinned
    int error = WRS_OK;
};

}  // namespace wrs

struct wrs_server {
    int device = 0;
    uint64_t budget = 0, resident = 0, transient = 0, peak = 0;
    uint32_t max_inflight = 2;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<wrs::Request *> queue;
    std::unordered_map<uint64_t, wrs::Request *> reqs;
    std::unordered_map<uint64_t, wrs::TableRec> tables;
    std::deque<wrs::Step *> inflight;
    std::vector<wrs::Slot> slots;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    cudaStream_t s_build = nullptr, s_sample = nullptr;
    cudaMemPool_t pool = nullptr;
    // stats
    std::vector<double> lat_ms;
    uint64_t n_build = 0, n_sample = 0, n_release = 0, n_error = 0, steps = 0, step_reqs = 0;
    uint64_t items_built = 0, samples_drawn = 0;
    double t_first = 0, t_last = 0;

    void run();
    void retire();
    bool launch_step();
    void finish(wrs::Request *r, int status, double t);
};

using namespace wrs;

void wrs_server::finish(Request *r, int status, double t) {
    r->status = status;
    r->t_done = t;
    r->done = true;
    lat_ms.push_back((r->t_done - r->t_submit) * 1e3);
    if (status != WRS_OK) ++n_error;
    if (r->kind == K_BUILD) ++n_build;
    else if (r->kind == K_SAMPLE) ++n_sample;
    else ++n_release;
    t_last = t;
    cv_done.notify_all();   // called with mu held; wakes wrs_server_wait
}

void wrs_server::retire() {
    for (;;) {
        Step *st = nullptr;
        {
            std::lock_guard<std::mutex> lk(mu);
            if (inflight.empty()) return;
            st = inflight.front();
        }
        cudaError_t q = cudaEventQuery(st->done);
        if (q == cudaErrorNotReady) return;
        int err = st->error != WRS_OK ? st->error : cuda_status(q);
        double t = now_s();
        std::lock_guard<std::mutex> lk(mu);
        inflight.pop_front();
        for (size_t k = 0; k < st->tables.size(); ++k) {
            TableRec &tr = tables[st->tables[k]];
            const wrs_table_summary &s = st->summ[k];
            tr.built = true;
            tr.status = err != WRS_OK ? err : s.status;
            tr.W = s.W;
            tr.nl = s.nl;
            tr.nh = s.nh;
            if (tr.status == WRS_OK) items_built += tr.n;
        }
        for (size_t k = 0; k < st->ltables.size(); ++k) {
            TableRec &tr = tables[st->ltables[k]];
            const wrs_build_info &b = st->linfo[k];
            tr.built = true;
            tr.status = err != WRS_OK ? err : b.status;
            tr.W = b.W;
            tr.nl = b.nl;
            tr.nh = b.nh;
            if (tr.status == WRS_OK) items_built += tr.n;
        }
        for (Request *r : st->reqs) {
            int status = err;
            if (status == WRS_OK) {
                if (r->kind == K_BUILD) {
                    status = tables[r->id].status;
                } else if (r->kind == K_SAMPLE) {
                    // the table may have failed in this or an earlier step
                    const TableRec &tr = tables[r->table];
                    status = (tr.built && tr.status != WRS_OK) ? tr.status : r->status;
                }
            }
            if (r->kind == K_SAMPLE && status == WRS_OK) {
                if (!r->out_dev)
                    memcpy(r->out, slots[st->slot].pin_out + r->stage_off, r->count * 4);
                samples_drawn += r->count;
            }
            finish(r, status, t);
        }
        // failed builds give their memory back
        for (int pass = 0; pass < 2; ++pass) {
            for (uint64_t id : pass ? st->ltables : st->tables) {
                TableRec &tr = tables[id];
                if (tr.status != WRS_OK && !tr.gone) {
                    tr.gone = true;
                    cudaFreeAsync(tr.rows, s_sample);
                    resident -= tr.bytes;
                }
            }
        }
        if (st->scratch) cudaFreeAsync(st->scratch, s_sample);
        for (void *p : st->lscratch) cudaFreeAsync(p, s_sample);
        transient -= st->scratch_bytes;
        slots[st->slot].busy = false;
        cudaEventDestroy(st->done);
        if (st->built) cudaEventDestroy(st->built);
        delete st;
        cv_done.notify_all();
    }
}

bool wrs_server::launch_step() {
    int slot = -1;
    std::vector<Request *> builds, large, samples, releases;
    uint64_t build_items = 0, sample_total = 0, host_samples = 0, scratch = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (queue.empty() || inflight.size() >= max_inflight) return false;
        for (size_t k = 0; k < slots.size(); ++k)
            if (!slots[k].busy) { slot = (int)k; break; }
        if (slot < 0) return false;
        bool builds_blocked = false;
        std::deque<Request *> keep;
        double t = now_s();
        uint32_t taken = 0;
        while (!queue.empty()) {
            Request *r = queue.front();
            queue.pop_front();
            if (taken >= kMaxReqPerStep) { keep.push_back(r); continue; }
            if (r->kind == K_BUILD) {
                // transient: weights + l/h array (batched), or weights + the
                // single-table workspace (large)
                uint64_t rows_b = 8 * r->n,
                         scr = r->n >= kLargeBuild
                                   ? 4 * r->n + make_layout(r->n, kLargeSection).total + 4096
                                   : 12 * r->n + 4096;
                if (rows_b + scr > budget) { finish(r, WRS_ENOMEM, t); continue; }
                if (builds_blocked || resident + transient + scratch + rows_b + scr > budget) {
                    builds_blocked = true;   // keep arrival order among builds
                    keep.push_back(r);
                    continue;
                }
                scratch += scr;
                resident += rows_b;
                TableRec tr;
                tr.n = r->n;
                tr.bytes = rows_b;
                tables[r->id] = tr;
                if (r->n >= kLargeBuild) {
                    large.push_back(r);
                } else {
                    builds.push_back(r);
                    build_items += r->n;
                }
                ++taken;
            } else {
                auto it = tables.find(r->table);
                if (it == tables.end() || it->second.gone) {
                    // its build may still be waiting for memory: keep it queued
                    bool queued_build = false;
                    for (Request *q2 : keep)
                        if (q2->kind == K_BUILD && q2->id == r->table) queued_build = true;
                    for (Request *q2 : queue)
                        if (q2->kind == K_BUILD && q2->id == r->table) queued_build = true;
                    if (queued_build) { keep.push_back(r); continue; }
                    finish(r, WRS_ENOTFOUND, t);
                    continue;
                }
                if (it->second.built && it->second.status != WRS_OK) {
                    finish(r, it->second.status, t);
                    continue;
                }
                if (r->kind == K_SAMPLE) {
                    samples.push_back(r);
                    sample_total += r->count;
                    if (!r->out_dev) {
                        r->stage_off = host_samples;
                        host_samples += r->count;
                    }
                } else {
                    it->second.gone = true;   // later requests for it fail
                    releases.push_back(r);
                }
                ++taken;
            }
        }
        queue.swap(keep);
        if (builds.empty() && large.empty() && samples.empty() && releases.empty()) return false;
        slots[slot].busy = true;
        transient += scratch;
        peak = std::max(peak, resident + transient);
    }
    Step *st = new Step();
    st->slot = slot;
    st->scratch_bytes = scratch;
    cudaEventCreateWithFlags(&st->done, cudaEventDisableTiming);
    cudaError_t e = cudaSuccess;
    Slot &sl = slots[slot];
    // pinned staging: offsets, row pointers, summaries, request descriptors
    const uint32_t nb = (uint32_t)builds.size(), ns = (uint32_t)samples.size();
    const uint32_t nlg = (uint32_t)large.size();
    uint64_t need_pin = align_up(8 * (nb + 1), 64) + align_up(8 * nb, 64) +
                        align_up(sizeof(wrs_table_summary) * nb, 64) +
                        align_up(sizeof(SampleReq) * ns, 64) + align_up(4 * (ns + 1), 64) +
                        align_up(sizeof(wrs_build_info) * nlg, 64);
    if (need_pin > sl.pin_bytes) {
        if (sl.pin) cudaFreeHost(sl.pin);
        sl.pin_bytes = std::max<uint64_t>(need_pin, 1 << 20);
        e = cudaMallocHost((void **)&sl.pin, sl.pin_bytes);
    }
    if (!e && host_samples * 4 > sl.pin_out_bytes) {
        if (sl.pin_out) cudaFreeHost(sl.pin_out);
        sl.pin_out_bytes = std::max<uint64_t>(host_samples * 4, 16 << 20);
        e = cudaMallocHost((void **)&sl.pin_out, sl.pin_out_bytes);
    }
    unsigned char *pp = sl.pin;
    uint64_t *h_off = (uint64_t *)pp;
    pp += align_up(8 * (nb + 1), 64);
    wrs_row **h_rowp = (wrs_row **)pp;
    pp += align_up(8 * nb, 64);
    st->summ = (wrs_table_summary *)pp;
    pp += align_up(sizeof(wrs_table_summary) * nb, 64);
    SampleReq *h_req = (SampleReq *)pp;
    pp += align_up(sizeof(SampleReq) * ns, 64);
    uint32_t *h_chunk = (uint32_t *)pp;
    pp += align_up(4 * (ns + 1), 64);
    st->linfo = (wrs_build_info *)pp;
    // device scratch for the step
    uint64_t dev_bytes = 256 + align_up(4 * build_items, 256) + align_up(8 * build_items, 256) +
                         align_up(8 * (nb + 1), 256) + align_up(8 * nb, 256) +
                         align_up(sizeof(wrs_table_summary) * nb, 256) +
                         align_up(sizeof(SampleReq) * ns, 256) + align_up(4 * (ns + 1), 256) +
                         align_up(4 * host_samples, 256) +
                         align_up(sizeof(wrs_build_info) * nlg, 256);
    unsigned char *d = nullptr;
    if (!e) e = cudaMallocFromPoolAsync((void **)&d, dev_bytes, pool, s_build);
    st->scratch = d;
    unsigned char *dp = d;
    auto take = [&](uint64_t b) {
        unsigned char *p = dp;
        dp += align_up(b, 256);
        return p;
    };
    uint32_t *d_counter = (uint32_t *)take(256);
    float *d_w = (float *)take(4 * build_items);
    Entry *d_lh = (Entry *)take(8 * build_items);
    uint64_t *d_off = (uint64_t *)take(8 * (nb + 1));
    wrs_row **d_rowp = (wrs_row **)take(8 * nb);
    wrs_table_summary *d_summ = (wrs_table_summary *)take(sizeof(wrs_table_summary) * nb);
    SampleReq *d_req = (SampleReq *)take(sizeof(SampleReq) * ns);
    uint32_t *d_chunk = (uint32_t *)take(4 * (ns + 1));
    uint32_t *d_stage = (uint32_t *)take(4 * host_samples);
    wrs_build_info *d_linfo = (wrs_build_info *)take(sizeof(wrs_build_info) * nlg);
    // ---- large builds: the single-table pipeline, one after another
    for (uint32_t k = 0; k < nlg && !e; ++k) {
        Request *r = large[k];
        const Layout L = make_layout(r->n, kLargeSection);
        uint64_t bytes;
        {
            std::lock_guard<std::mutex> lk(mu);
            bytes = tables[r->id].bytes;
        }
        wrs_row *rp = nullptr;
        unsigned char *lw = nullptr;
        e = cudaMallocFromPoolAsync((void **)&rp, bytes, pool, s_build);
        if (!e) e = cudaMallocFromPoolAsync((void **)&lw, align_up(4 * r->n, 256) + L.total, pool,
                                            s_build);
        {
            std::lock_guard<std::mutex> lk(mu);
            tables[r->id].rows = rp;
        }
        st->ltables.push_back(r->id);
        if (lw) st->lscratch.push_back(lw);
        if (e) break;
        float *wk = (float *)lw;
        unsigned char *ws = lw + align_up(4 * r->n, 256);
        e = cudaMemcpyAsync(wk, r->w, 4 * r->n,
                            r->w_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s_build);
        if (!e) e = launch_total(wk, r->n, ws, L, s_build);
        if (!e) e = launch_partition(wk, r->n, ws, L, s_build);
        if (!e) e = launch_split(r->n, ws, L, kLargeSection, WRS_SPLIT_PARY, s_build);
        if (!e) e = launch_pack(r->n, rp, ws, L, kLargeSection, s_build);
        if (!e) e = launch_info(ws, L, d_linfo + k, s_build);
    }
    if (!e && nlg)
        e = cudaMemcpyAsync(st->linfo, d_linfo, sizeof(wrs_build_info) * nlg,
                            cudaMemcpyDeviceToHost, s_build);
    // ---- builds
    if (!e && nb) {
        h_off[0] = 0;
        for (uint32_t k = 0; k < nb; ++k) {
            Request *r = builds[k];
            wrs_row *rp = nullptr;
            uint64_t bytes;
            {
                std::lock_guard<std::mutex> lk(mu);
                bytes = tables[r->id].bytes;
            }
            if (!e) e = cudaMallocFromPoolAsync((void **)&rp, bytes, pool, s_build);
            {
                std::lock_guard<std::mutex> lk(mu);
                tables[r->id].rows = rp;
            }
            h_rowp[k] = rp;
            if (!e)
                e = cudaMemcpyAsync(d_w + h_off[k], r->w, 4 * r->n,
                                    r->w_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    s_build);
            h_off[k + 1] = h_off[k] + r->n;
            st->tables.push_back(r->id);
        }
        if (!e) e = cudaMemcpyAsync(d_off, h_off, 8 * (nb + 1), cudaMemcpyHostToDevice, s_build);
        if (!e) e = cudaMemcpyAsync(d_rowp, h_rowp, 8 * nb, cudaMemcpyHostToDevice, s_build);
        if (!e)
            e = launch_build_batched(d_w, d_off, nb, nullptr, d_counter, d_lh, nullptr, d_rowp,
                                     d_summ, nullptr, s_build);
        if (!e)
            e = cudaMemcpyAsync(st->summ, d_summ, sizeof(wrs_table_summary) * nb,
                                cudaMemcpyDeviceToHost, s_build);
    }
    if (!e && (nb || nlg)) {
        e = cudaEventCreateWithFlags(&st->built, cudaEventDisableTiming);
        if (!e) e = cudaEventRecord(st->built, s_build);
        std::lock_guard<std::mutex> lk(mu);
        for (uint32_t k = 0; k < nb; ++k) tables[builds[k]->id].ready = st->built;
        for (uint32_t k = 0; k < nlg; ++k) tables[large[k]->id].ready = st->built;
    }
    // ---- samples (wait on the GPU for tables still being built)
    if (!e && ns) {
        std::vector<cudaEvent_t> waits;
        uint32_t blocks = 0;
        std::unique_lock<std::mutex> lk(mu);
        for (uint32_t k = 0; k < ns; ++k) {
            Request *r = samples[k];
            TableRec &tr = tables[r->table];
            if (!tr.built && tr.ready &&
                std::find(waits.begin(), waits.end(), tr.ready) == waits.end())
                waits.push_back(tr.ready);
            SampleReq q;
            q.rows = tr.rows;
            q.n = tr.n;
            q.count = r->count;
            q.out = r->out_dev ? r->out : d_stage + r->stage_off;
            q.k0 = (uint32_t)r->seed;
            q.k1 = (uint32_t)(r->seed >> 32);
            q.slo = r->slo;
            q.shi = WRS_TAG_NAIVE;
            h_req[k] = q;
            h_chunk[k] = blocks;
            blocks += (uint32_t)((r->count + kReqChunkH - 1) / kReqChunkH);
        }
        h_chunk[ns] = blocks;
        lk.unlock();
        for (cudaEvent_t ev : waits)
            if (!e) e = cudaStreamWaitEvent(s_sample, ev, 0);
        if (!e)
            e = cudaMemcpyAsync(d_req, h_req, sizeof(SampleReq) * ns, cudaMemcpyHostToDevice,
                                s_sample);
        if (!e)
            e = cudaMemcpyAsync(d_chunk, h_chunk, 4 * (ns + 1), cudaMemcpyHostToDevice, s_sample);
        if (!e) e = launch_sample_requests(d_req, d_chunk, ns, blocks, s_sample);
        if (!e && host_samples)
            e = cudaMemcpyAsync(sl.pin_out, d_stage, 4 * host_samples, cudaMemcpyDeviceToHost,
                                s_sample);
    }
    // ---- releases (after every earlier use of the table, in stream order)
    if (!e && !releases.empty()) {
        std::lock_guard<std::mutex> lk(mu);
        for (Request *r : releases) {
            TableRec &tr = tables[r->table];
            if (tr.ready && !tr.built) e = cudaStreamWaitEvent(s_sample, tr.ready, 0);
            if (!e) e = cudaFreeAsync(tr.rows, s_sample);
            resident -= tr.bytes;
            tr.rows = nullptr;
        }
    }
    // the step is done when both streams have passed it
    if (!e && st->built) e = cudaStreamWaitEvent(s_sample, st->built, 0);
    if (!e) e = cudaEventRecord(st->done, s_sample);
    if (e) {
        st->error = cuda_status(e);
        cudaStreamSynchronize(s_build);
        cudaStreamSynchronize(s_sample);
        cudaEventRecord(st->done, s_sample);
    }
    std::lock_guard<std::mutex> lk(mu);
    st->reqs = builds;
    st->reqs.insert(st->reqs.end(), large.begin(), large.end());
    st->reqs.insert(st->reqs.end(), samples.begin(), samples.end());
    st->reqs.insert(st->reqs.end(), releases.begin(), releases.end());
    ++steps;
    step_reqs += st->reqs.size();
    inflight.push_back(st);
    return true;
}

void wrs_server::run() {
    cudaSetDevice(device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait_for(lk, std::chrono::microseconds(100), [&] {
                return stop || !queue.empty() || !inflight.empty();
            });
            if (stop && queue.empty() && inflight.empty()) return;
        }
        retire();
        while (launch_step()) {
        }
        bool idle;
        {
            std::lock_guard<std::mutex> lk(mu);
            idle = queue.empty() || inflight.size() >= max_inflight;
        }
        if (idle) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

extern "C" {

int wrs_server_create(uint64_t hbm_budget, uint32_t max_inflight, wrs_server **out) {
    if (!out || hbm_budget == 0 || max_inflight == 0 || max_inflight > 64) return WRS_EINVAL;
    wrs_server *s = new wrs_server();
    cudaError_t e = cudaGetDevice(&s->device);
    s->budget = hbm_budget;
    s->max_inflight = max_inflight;
    s->slots.resize(max_inflight);
    if (!e) e = cudaStreamCreateWithFlags(&s->s_build, cudaStreamNonBlocking);
    if (!e) e = cudaStreamCreateWithFlags(&s->s_sample, cudaStreamNonBlocking);
    if (!e) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = s->device;
        e = cudaMemPoolCreate(&s->pool, &props);
        if (!e) {
            uint64_t keep = ~0ull;   // keep freed memory in the pool
            e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (e) {
        int rc = cuda_status(e);
        if (s->s_build) cudaStreamDestroy(s->s_build);
        if (s->s_sample) cudaStreamDestroy(s->s_sample);
        if (s->pool) cudaMemPoolDestroy(s->pool);
        delete s;
        return rc;
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return WRS_OK;
}

static int submit(wrs_server *s, Request *r, uint64_t *ticket) {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->t_submit = now_s();
    if (s->t_first == 0) s->t_first = r->t_submit;
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    *ticket = r->id;
    s->cv_work.notify_one();
    return WRS_OK;
}

int wrs_server_submit_build(wrs_server *s, const float *w, uint64_t n, int w_on_device,
                            uint64_t *ticket) {
    if (!s || !w || !ticket || n == 0 || n > kMaxServerItems) return WRS_EINVAL;
    Request *r = new Request();
    r->kind = K_BUILD;
    r->w = w;
    r->n = n;
    r->w_dev = w_on_device;
    return submit(s, r, ticket);
}

int wrs_server_submit_sample(wrs_server *s, uint64_t table, uint64_t count, uint64_t seed,
                             uint32_t stream_lo, uint32_t *out, int out_on_device,
                             uint64_t *ticket) {
    if (!s || !ticket || (count && !out)) return WRS_EINVAL;
    Request *r = new Request();
    r->kind = K_SAMPLE;
    r->table = table;
    r->count = count;
    r->seed = seed;
    r->slo = stream_lo;
    r->out = out;
    r->out_dev = out_on_device;
    return submit(s, r, ticket);
}

int wrs_server_submit_release(wrs_server *s, uint64_t table, uint64_t *ticket) {
    if (!s || !ticket) return WRS_EINVAL;
    Request *r = new Request();
    r->kind = K_RELEASE;
    r->table = table;
    return submit(s, r, ticket);
}

int wrs_server_poll(wrs_server *s, uint64_t ticket, int *done, int *status) {
    if (!s || !done || !status) return WRS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return WRS_ENOTFOUND;
    *done = it->second->done;
    *status = it->second->status;
    return WRS_OK;
}

int wrs_server_wait(wrs_server *s, uint64_t ticket, int *status) {
    if (!s || !status) return WRS_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return WRS_ENOTFOUND;
    Request *r = it->second;
    s->cv_done.wait(lk, [&] { return r->done; });
    *status = r->status;
    return WRS_OK;
}

int wrs_server_table(wrs_server *s, uint64_t table, const wrs_row **d_rows, uint64_t *n,
                     double *W) {
    if (!s || !d_rows || !n) return WRS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tables.find(table);
    if (it == s->tables.end() || it->second.gone || !it->second.built) return WRS_ENOTFOUND;
    *d_rows = it->second.rows;
    *n = it->second.n;
    if (W) *W = it->second.W;
    return WRS_OK;
}

int wrs_server_export(wrs_server *s, uint64_t table, wrs_row *dst, int dst_on_device) {
    if (!s || !dst) return WRS_EINVAL;
    const wrs_row *rows;
    uint64_t n;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->tables.find(table);
        if (it == s->tables.end() || it->second.gone || !it->second.built) return WRS_ENOTFOUND;
        rows = it->second.rows;
        n = it->second.n;
    }
    // the copy is ordered after every earlier use of the table on the
    // sample stream; the caller then owns a snapshot of the rows
    cudaError_t e = cudaMemcpyAsync(dst, rows, n * sizeof(wrs_row),
                                    dst_on_device ? cudaMemcpyDeviceToDevice
                                                  : cudaMemcpyDeviceToHost,
                                    s->s_sample);
    if (!e) e = cudaStreamSynchronize(s->s_sample);
    return cuda_status(e);
}

int wrs_server_stats(wrs_server *s, wrs_server_statistics *out) {
    if (!s || !out) return WRS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof *out);
    out->completed = s->lat_ms.size();
    out->builds = s->n_build;
    out->samples = s->n_sample;
    out->releases = s->n_release;
    out->errors = s->n_error;
    out->items_built = s->items_built;
    out->samples_drawn = s->samples_drawn;
    out->steps = s->steps;
    out->mean_step_requests = s->steps ? (double)s->step_reqs / s->steps : 0.0;
    out->resident_bytes = s->resident;
    out->peak_bytes = s->peak;
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            size_t k = (size_t)(p * (v.size() - 1) + 0.5);
            return v[std::min(k, v.size() - 1)];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_ms = sum / v.size();
    }
    out->wall_s = s->t_last > s->t_first ? s->t_last - s->t_first : 0.0;
    return WRS_OK;
}

int wrs_server_destroy(wrs_server *s) {
    if (!s) return WRS_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    s->worker.join();
    cudaSetDevice(s->device);
    for (auto &kv : s->tables)
        if (!kv.second.gone && kv.second.rows) cudaFreeAsync(kv.second.rows, s->s_sample);
    cudaStreamSynchronize(s->s_sample);
    cudaStreamSynchronize(s->s_build);
    for (auto &sl : s->slots) {
        if (sl.pin) cudaFreeHost(sl.pin);
        if (sl.pin_out) cudaFreeHost(sl.pin_out);
    }
    for (auto &kv : s->reqs) delete kv.second;
    cudaStreamDestroy(s->s_build);
    cudaStreamDestroy(s->s_sample);
    cudaMemPoolDestroy(s->pool);
    delete s;
    return WRS_OK;
}

}  // extern "C"
