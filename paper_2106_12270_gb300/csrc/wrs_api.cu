// wrs_api.cu - the C ABI (include/wrs.h): argument checks on the host, then
// kernel launches on the caller's stream.  No torch types, no exceptions.
#include <string.h>

#include <algorithm>
#include <numeric>
#include <map>
#include <mutex>
#include <vector>

#include "wrs_internal.cuh"

namespace wrs {
cudaError_t launch_total(const float *, uint64_t, unsigned char *, const Layout &, cudaStream_t);
cudaError_t launch_partition(const float *, uint64_t, unsigned char *, const Layout &,
                             cudaStream_t);
cudaError_t launch_split(uint64_t, unsigned char *, const Layout &, uint32_t, uint32_t,
                         cudaStream_t);
cudaError_t launch_pack(uint64_t, wrs_row *, unsigned char *, const Layout &, uint32_t,
                        cudaStream_t);
cudaError_t launch_info(unsigned char *, const Layout &, wrs_build_info *, cudaStream_t);
cudaError_t launch_sample_naive(const wrs_row *, uint64_t, uint64_t, uint64_t, uint64_t,
                                uint32_t, uint32_t, uint32_t *, cudaStream_t);
cudaError_t launch_sample_sectioned(const wrs_row *, uint64_t, uint64_t, uint64_t, uint32_t,
                                    uint64_t, uint64_t *, uint64_t *, uint32_t *, cudaStream_t);

cudaError_t launch_sample_batched(const wrs_row *, const uint64_t *, uint32_t, const uint64_t *,
                                  uint64_t, uint32_t *, cudaStream_t);
cudaError_t launch_random_gather(const void *, uint64_t, uint64_t, uint64_t, int, uint32_t,
                                 uint32_t, uint32_t *, cudaStream_t);
cudaError_t launch_philox_rate(uint64_t, uint64_t, uint32_t *, cudaStream_t);
cudaError_t launch_pack_variant(const float *, uint64_t, wrs_row *, unsigned char *, const Layout &,
                                uint32_t, uint32_t, cudaStream_t);

uint64_t prec_workspace_bytes(uint64_t n, uint32_t S);
cudaError_t launch_prec_split_pack(uint64_t n, wrs_row *d_rows, unsigned char *ws, const Layout &L,
                                   unsigned char *pws, uint32_t S, uint32_t prec, cudaStream_t st);

struct PlusLayout;
uint64_t plus_workspace_bytes(uint64_t n, uint32_t S);
cudaError_t launch_build_plus_ws(const float *d_w, uint64_t n, wrs_row *d_rows, unsigned char *ws,
                                 uint32_t S, uint32_t split_method, uint32_t min_items,
                                 wrs_build_info *d_info, uint64_t *h_rest, cudaStream_t st);

thread_local int g_last_cuda = 0;

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return WRS_OK;
    g_last_cuda = (int)e;
    return e == cudaErrorMemoryAllocation ? WRS_ENOMEM : WRS_ECUDA;
}

constexpr uint64_t kMaxN = 0x7fffffffull;

int resolve_cfg(const wrs_config *in, wrs_config *out) {
    wrs_config_default(out);
    if (in) *out = *in;
    if (out->section_size < 256 || out->section_size > 8192 || out->section_size % 256)
        return WRS_EINVAL;
    if (out->split_method != WRS_SPLIT_PARY && out->split_method != WRS_SPLIT_BINARY)
        return WRS_EINVAL;
    return WRS_OK;
}

// Common checks of the step calls; fills the layout.
static int prep(uint64_t n, const void *ws, uint64_t ws_bytes, const wrs_config *cfg,
                wrs_config *c, Layout *L) {
    if (n == 0 || n > kMaxN) return WRS_EINVAL;
    int rc = resolve_cfg(cfg, c);
    if (rc) return rc;
    *L = make_layout(n, c->section_size);
    if (!ws || ((uintptr_t)ws & 255u) || ws_bytes < L->total) return WRS_EINVAL;
    return WRS_OK;
}

}  // namespace wrs

using namespace wrs;

extern "C" {

const char *wrs_strerror(int s) {
    switch (s) {
        case WRS_OK: return "ok";
        case WRS_EINVAL: return "invalid argument or negative weight";
        case WRS_EZEROSUM: return "all weights are zero";
        case WRS_ENONFINITE: return "a weight is NaN or infinite";
        case WRS_ENOMEM: return "out of device memory or over budget";
        case WRS_ETIMEOUT: return "a bounded device wait gave up";
        case WRS_ECUDA: return "CUDA runtime error";
        case WRS_EBUSY: return "busy: no room right now";
        case WRS_ENOTFOUND: return "unknown ticket";
        default: return "unknown status";
    }
}

int wrs_last_cuda_error(void) { return g_last_cuda; }

int wrs_abi_version(void) { return 2; }

void wrs_config_default(wrs_config *cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->section_size = 1024;
    cfg->split_method = WRS_SPLIT_PARY;
}

int wrs_build_workspace_bytes(uint64_t n, const wrs_config *cfg, uint64_t *bytes) {
    wrs_config c;
    if (!bytes || n == 0 || n > kMaxN) return WRS_EINVAL;
    int rc = resolve_cfg(cfg, &c);
    if (rc) return rc;
    *bytes = make_layout(n, c.section_size).total;
    return WRS_OK;
}

int wrs_build_layout(uint64_t n, const wrs_config *cfg, wrs_layout *out) {
    wrs_config c;
    if (!out || n == 0 || n > kMaxN) return WRS_EINVAL;
    int rc = resolve_cfg(cfg, &c);
    if (rc) return rc;
    Layout L = make_layout(n, c.section_size);
    out->lh = L.lh;
    out->ckl = L.ckl;
    out->ckh = L.ckh;
    out->seg_pre = L.seg_pre;
    out->splits = L.splits;
    out->sections = L.sections;
    out->total_bytes = L.total;
    return WRS_OK;
}

int wrs_step_total(const float *d_w, uint64_t n, void *d_ws, uint64_t ws_bytes,
                   const wrs_config *cfg, void *stream) {
    wrs_config c;
    Layout L;
    int rc = prep(n, d_ws, ws_bytes, cfg, &c, &L);
    if (rc) return rc;
    if (!d_w || ((uintptr_t)d_w & 3u)) return WRS_EINVAL;
    return cuda_status(launch_total(d_w, n, (unsigned char *)d_ws, L, (cudaStream_t)stream));
}

int wrs_step_partition(const float *d_w, uint64_t n, void *d_ws, uint64_t ws_bytes,
                       const wrs_config *cfg, void *stream) {
    wrs_config c;
    Layout L;
    int rc = prep(n, d_ws, ws_bytes, cfg, &c, &L);
    if (rc) return rc;
    if (!d_w || ((uintptr_t)d_w & 3u)) return WRS_EINVAL;
    return cuda_status(launch_partition(d_w, n, (unsigned char *)d_ws, L, (cudaStream_t)stream));
}

int wrs_step_split(uint64_t n, void *d_ws, uint64_t ws_bytes, const wrs_config *cfg,
                   void *stream) {
    wrs_config c;
    Layout L;
    int rc = prep(n, d_ws, ws_bytes, cfg, &c, &L);
    if (rc) return rc;
    return cuda_status(launch_split(n, (unsigned char *)d_ws, L, c.section_size,
                                    c.split_method, (cudaStream_t)stream));
}

int wrs_step_pack(uint64_t n, wrs_row *d_rows, void *d_ws, uint64_t ws_bytes,
                  const wrs_config *cfg, void *stream) {
    wrs_config c;
    Layout L;
    int rc = prep(n, d_ws, ws_bytes, cfg, &c, &L);
    if (rc) return rc;
    if (!d_rows || ((uintptr_t)d_rows & 7u)) return WRS_EINVAL;
    return cuda_status(
        launch_pack(n, d_rows, (unsigned char *)d_ws, L, c.section_size, (cudaStream_t)stream));
}

int wrs_step_info(uint64_t n, void *d_ws, uint64_t ws_bytes, const wrs_config *cfg,
                  wrs_build_info *d_info, void *stream) {
    wrs_config c;
    Layout L;
    int rc = prep(n, d_ws, ws_bytes, cfg, &c, &L);
    if (rc) return rc;
    if (!d_info) return WRS_EINVAL;
    return cuda_status(launch_info((unsigned char *)d_ws, L, d_info, (cudaStream_t)stream));
}

int wrs_build_rows(const float *d_w, uint64_t n, wrs_row *d_rows, void *d_ws, uint64_t ws_bytes,
                   const wrs_config *cfg, wrs_build_info *d_info, void *stream) {
    wrs_config c;
    Layout L;
    int rc = prep(n, d_ws, ws_bytes, cfg, &c, &L);
    if (rc) return rc;
    if (!d_w || ((uintptr_t)d_w & 3u) || !d_rows || ((uintptr_t)d_rows & 7u) || !d_info)
        return WRS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *ws = (unsigned char *)d_ws;
    cudaError_t e = launch_total(d_w, n, ws, L, st);
    if (!e) e = launch_partition(d_w, n, ws, L, st);
    if (!e) e = launch_split(n, ws, L, c.section_size, c.split_method, st);
    if (!e) e = launch_pack(n, d_rows, ws, L, c.section_size, st);
    if (!e) e = launch_info(ws, L, d_info, st);
    return cuda_status(e);
}

int wrs_build_plus_workspace_bytes(uint64_t n, const wrs_config *cfg, uint64_t *bytes) {
    if (!bytes || n == 0 || n > kMaxN) return WRS_EINVAL;
    wrs_config c;
    int rc = resolve_cfg(cfg, &c);
    if (rc) return rc;
    *bytes = plus_workspace_bytes(n, c.section_size);
    return WRS_OK;
}

int wrs_build_rows_plus(const float *d_w, uint64_t n, wrs_row *d_rows, void *d_ws,
                        uint64_t ws_bytes, const wrs_config *cfg, uint32_t min_items,
                        wrs_build_info *d_info, uint64_t *greedy_items, void *stream) {
    if (n == 0 || n > kMaxN) return WRS_EINVAL;
    wrs_config c;
    int rc = resolve_cfg(cfg, &c);
    if (rc) return rc;
    if (!d_ws || ((uintptr_t)d_ws & 255u) || ws_bytes < plus_workspace_bytes(n, c.section_size))
        return WRS_EINVAL;
    if (!d_w || ((uintptr_t)d_w & 3u) || !d_rows || ((uintptr_t)d_rows & 7u) || !d_info)
        return WRS_EINVAL;
    uint64_t greedy = 0;
    cudaError_t e = launch_build_plus_ws(d_w, n, d_rows, (unsigned char *)d_ws, c.section_size,
                                         c.split_method, min_items, d_info, &greedy,
                                         (cudaStream_t)stream);
    if (greedy_items) *greedy_items = e ? 0 : greedy;
    return cuda_status(e);
}

// Host-buffer build: [build workspace][weights][rows][summary], each region
// 256-byte aligned.
static uint64_t host_ws_regions(uint64_t build_total, uint64_t n, uint64_t *w_off, uint64_t *r_off,
                                uint64_t *i_off) {
    *w_off = align_up(build_total, 256);
    *r_off = *w_off + align_up(4 * n, 256);
    *i_off = *r_off + align_up(8 * n, 256);
    return *i_off + align_up(sizeof(wrs_build_info), 256);
}

int wrs_build_host_workspace_bytes(uint64_t n, const wrs_config *cfg, uint64_t *bytes) {
    uint64_t b = 0;
    int rc = wrs_build_workspace_bytes(n, cfg, &b);
    if (rc) return rc;
    uint64_t wo, ro, io;
    *bytes = host_ws_regions(b, n, &wo, &ro, &io);
    return WRS_OK;
}

int wrs_build_rows_host(const float *h_w, uint64_t n, wrs_row *h_rows, void *d_ws,
                        uint64_t ws_bytes, const wrs_config *cfg, wrs_build_info *h_info,
                        void *stream) {
    uint64_t b = 0;
    int rc = wrs_build_workspace_bytes(n, cfg, &b);
    if (rc) return rc;
    if (!h_w || !h_rows || !h_info || !d_ws || ((uintptr_t)d_ws & 255u)) return WRS_EINVAL;
    uint64_t wo, ro, io;
    if (ws_bytes < host_ws_regions(b, n, &wo, &ro, &io)) return WRS_EINVAL;
    unsigned char *ws = (unsigned char *)d_ws;
    float *d_w = reinterpret_cast<float *>(ws + wo);
    wrs_row *d_rows = reinterpret_cast<wrs_row *>(ws + ro);
    wrs_build_info *d_info = reinterpret_cast<wrs_build_info *>(ws + io);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(d_w, h_w, 4 * n, cudaMemcpyHostToDevice, st);
    if (e) return cuda_status(e);
    rc = wrs_build_rows(d_w, n, d_rows, d_ws, b, cfg, d_info, stream);
    if (rc) return rc;
    e = cudaMemcpyAsync(h_rows, d_rows, 8 * n, cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaMemcpyAsync(h_info, d_info, sizeof(wrs_build_info), cudaMemcpyDeviceToHost, st);
    return cuda_status(e);
}

int wrs_sample_rows(const wrs_row *d_rows, uint64_t n, uint64_t first, uint64_t count,
                    uint64_t seed, uint32_t stream_lo, uint32_t stream_hi, uint32_t *d_out,
                    void *stream) {
    if (n == 0 || n > kMaxN || !d_rows || ((uintptr_t)d_rows & 7u)) return WRS_EINVAL;
    if (count && (!d_out || ((uintptr_t)d_out & 3u))) return WRS_EINVAL;
    if (first + count < first) return WRS_EINVAL;
    return cuda_status(launch_sample_naive(d_rows, n, first, count, seed, stream_lo, stream_hi,
                                           d_out, (cudaStream_t)stream));
}

int wrs_sample_sections(uint64_t n, uint32_t section_rows, uint64_t *nsec) {
    if (!nsec || n == 0 || n > kMaxN || section_rows == 0) return WRS_EINVAL;
    *nsec = (n + section_rows - 1) / section_rows;
    return WRS_OK;
}

int wrs_sample_sectioned_rows(const wrs_row *d_rows, uint64_t n, uint64_t count, uint64_t seed,
                              uint32_t mode, uint32_t section_rows, uint64_t *d_counts,
                              uint64_t *d_offsets, uint32_t *d_out, void *stream) {
    uint64_t nsec;
    int rc = wrs_sample_sections(n, section_rows, &nsec);
    if (rc) return rc;
    if (!d_rows || ((uintptr_t)d_rows & 7u) || !d_counts || !d_offsets) return WRS_EINVAL;
    if (((uintptr_t)d_counts & 7u) || ((uintptr_t)d_offsets & 7u)) return WRS_EINVAL;
    if (count && (!d_out || ((uintptr_t)d_out & 3u))) return WRS_EINVAL;
    if (mode < WRS_SAMPLE_CACHED || mode > WRS_SAMPLE_SMEM) return WRS_EINVAL;
    if (mode == WRS_SAMPLE_SMEM && section_rows > 24576) return WRS_EINVAL;
    if (nsec > 0x7fffffffull) return WRS_EINVAL;
    return cuda_status(launch_sample_sectioned(d_rows, n, count, seed, mode, nsec, d_counts,
                                               d_offsets, d_out, (cudaStream_t)stream));
}

int wrs_sample_auto_choice(uint64_t n, uint64_t count, uint32_t *mode, uint32_t *section_rows) {
    if (!mode || !section_rows || n == 0) return WRS_EINVAL;
    // measured on GB300 (sampler heat map over 2^16..2^27 rows and 2^16..2^28
    // draws): naive sampling wins while the table fits in L2 and the draws
    // per row are few.  From about half of L2 (2^23 rows = 64 MB) and 2^23
    // draws a sectioned mode pays: the shared-memory mode (4096-row
    // sections, each row's threshold converted once) from about 8 draws per
    // row, the cached mode (8192-row sections, rows read through L1) below.
    // Tables of 2^20+ rows with 128+ draws per row also take the
    // shared-memory mode; smaller tables have too few sections to fill the GPU.
    const bool big = n >= (1ull << 23) && count >= (1ull << 23);
    const bool dense = n >= (1ull << 20) && count / n >= 128;
    if ((big && count / n >= 8) || dense) {
        *mode = WRS_SAMPLE_SMEM;
        *section_rows = 4096u;
    } else if (big) {
        *mode = WRS_SAMPLE_CACHED;
        *section_rows = 8192u;
    } else {
        *mode = WRS_SAMPLE_NAIVE;
        *section_rows = 0u;
    }
    return WRS_OK;
}

int wrs_sample_auto_workspace_bytes(uint64_t n, uint64_t count, uint64_t *bytes) {
    if (!bytes) return WRS_EINVAL;
    uint32_t mode, rows;
    int rc = wrs_sample_auto_choice(n, count, &mode, &rows);
    if (rc) return rc;
    uint64_t nsec = 0;
    if (mode != WRS_SAMPLE_NAIVE) {
        rc = wrs_sample_sections(n, rows, &nsec);
        if (rc) return rc;
    }
    *bytes = 2 * align_up(8 * nsec, 256);
    return WRS_OK;
}

int wrs_sample_auto(const wrs_row *d_rows, uint64_t n, uint64_t count, uint64_t seed,
                    uint32_t *d_out, void *d_ws, uint64_t ws_bytes, uint32_t *mode_used,
                    void *stream) {
    uint32_t mode, rows;
    int rc = wrs_sample_auto_choice(n, count, &mode, &rows);
    if (rc) return rc;
    if (mode_used) *mode_used = mode;
    if (mode == WRS_SAMPLE_NAIVE)
        return wrs_sample_rows(d_rows, n, 0, count, seed, 0, WRS_TAG_NAIVE, d_out, stream);
    uint64_t nsec = 0;
    rc = wrs_sample_sections(n, rows, &nsec);
    if (rc) return rc;
    const uint64_t half = align_up(8 * nsec, 256);
    if (!d_ws || ((uintptr_t)d_ws & 255u) || ws_bytes < 2 * half) return WRS_EINVAL;
    unsigned char *ws = (unsigned char *)d_ws;
    return wrs_sample_sectioned_rows(d_rows, n, count, seed, mode, rows,
                                     reinterpret_cast<uint64_t *>(ws),
                                     reinterpret_cast<uint64_t *>(ws + half), d_out, stream);
}

int wrs_build_batched_workspace_bytes(uint64_t total, uint32_t ntab, uint64_t *bytes) {
    if (!bytes) return WRS_EINVAL;
    *bytes = batch_seg_layout(total, ntab).total;
    return WRS_OK;
}

int wrs_batch_order(const uint64_t *h_off, uint32_t ntab, uint32_t *h_order) {
    if (!h_off || (ntab && !h_order)) return WRS_EINVAL;
    std::vector<uint32_t> idx(ntab);
    std::iota(idx.begin(), idx.end(), 0u);
    std::stable_sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) {
        return h_off[a + 1] - h_off[a] > h_off[b + 1] - h_off[b];
    });
    std::copy(idx.begin(), idx.end(), h_order);
    return WRS_OK;
}

int wrs_batch_tuning_default(wrs_batch_tuning *t) {
    if (!t) return WRS_EINVAL;
    memset(t, 0, sizeof *t);   // threads 0: the segmented build
    return WRS_OK;
}

int wrs_build_batched_rows_tuned(const float *d_w, const uint64_t *d_off, uint32_t ntab,
                                 const uint32_t *d_order, wrs_row *d_rows, void *d_ws,
                                 uint64_t ws_bytes, wrs_table_summary *d_info,
                                 const wrs_batch_tuning *tuning, void *stream) {
    if (ntab == 0) return WRS_OK;
    if (!d_w || ((uintptr_t)d_w & 3u) || !d_off || ((uintptr_t)d_off & 7u) || !d_rows ||
        ((uintptr_t)d_rows & 7u) || !d_ws || ((uintptr_t)d_ws & 255u) || !d_info)
        return WRS_EINVAL;
    if (ws_bytes < 256) return WRS_EINVAL;
    if (tuning && !batch_tuning_valid(*tuning)) return WRS_EINVAL;
    unsigned char *ws = (unsigned char *)d_ws;
    if (!tuning || tuning->threads == 0) {
        // the segmented build: the largest item count whose layout fits
        // ws_bytes (the total is on the device; a table beyond it fails
        // with WRS_EINVAL in its summary)
        uint64_t lo = 0, hi = ws_bytes / sizeof(Entry);
        while (lo < hi) {
            const uint64_t mid = lo + (hi - lo + 1) / 2;
            if (batch_seg_layout(mid, ntab).total <= ws_bytes) lo = mid;
            else hi = mid - 1;
        }
        const BatchSegLayout L = batch_seg_layout(lo, ntab);
        if (L.total > ws_bytes) return WRS_EINVAL;
        return cuda_status(launch_build_batched_seg(d_w, d_off, ntab, d_order, ws, L, d_rows,
                                                    nullptr, d_info, (cudaStream_t)stream));
    }
    // the chunked kernel: one l/h entry per item after the counter; the total
    // is on the device, so the kernel trusts ws_bytes >= 256 + 8 * total
    return cuda_status(launch_build_batched(d_w, d_off, ntab, d_order,
                                            reinterpret_cast<uint32_t *>(ws),
                                            reinterpret_cast<Entry *>(ws + 256), d_rows, nullptr,
                                            d_info, tuning, (cudaStream_t)stream));
}

int wrs_build_batched_rows(const float *d_w, const uint64_t *d_off, uint32_t ntab,
                           const uint32_t *d_order, wrs_row *d_rows, void *d_ws, uint64_t ws_bytes,
                           wrs_table_summary *d_info, void *stream) {
    return wrs_build_batched_rows_tuned(d_w, d_off, ntab, d_order, d_rows, d_ws, ws_bytes, d_info,
                                        nullptr, stream);
}

}  // extern "C"

namespace {
std::mutex g_tune_mu;
std::map<std::pair<uint32_t, uint64_t>, wrs_batch_tuning> g_tune_cache;
}  // namespace

namespace wrs {
// The autotuner's choice for a batch shape, if it has timed one.
bool cached_batch_tuning(uint32_t ntab, uint64_t total, wrs_batch_tuning *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(std::make_pair(ntab, total));
    if (it == g_tune_cache.end()) return false;
    *out = it->second;
    return true;
}
}  // namespace wrs

extern "C" {

int wrs_batch_autotune(const float *d_w, const uint64_t *d_off, uint32_t ntab,
                       const uint32_t *d_order, wrs_row *d_rows, void *d_ws, uint64_t ws_bytes,
                       wrs_table_summary *d_info, void *stream, int force,
                       wrs_batch_tuning *best, wrs_batch_tuning *all, uint32_t *nall) {
    if (!best || ntab == 0) return WRS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t total = 0;
    cudaError_t e = cudaMemcpyAsync(&total, d_off + ntab, sizeof total, cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return cuda_status(e);
    const auto key = std::make_pair(ntab, total);
    if (!force) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *best = it->second;
            if (nall) *nall = 0;
            return WRS_OK;
        }
    }
    static const uint32_t kThreads[] = {256, 512};
    static const uint32_t kChunks[] = {512, 1024, 2048, 4096};
    std::vector<wrs_batch_tuning> cand;
    {
        wrs_batch_tuning x;   // the segmented build
        wrs_batch_tuning_default(&x);
        cand.push_back(x);
    }
    for (uint32_t t : kThreads)
        for (uint32_t c : kChunks) {
            wrs_batch_tuning x;
            wrs_batch_tuning_default(&x);
            x.threads = t;
            x.chunk = c;
            cand.push_back(x);
        }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    // warm-up (first launches of each tiling configure its kernel)
    int rc = WRS_OK;
    for (auto &x : cand) {
        if (rc || e) break;
        rc = wrs_build_batched_rows_tuned(d_w, d_off, ntab, d_order, d_rows, d_ws, ws_bytes, d_info,
                                          &x, stream);
    }
    for (auto &x : cand) {
        float bestms = 0.f;
        for (int rep = 0; rep < 2 && !rc && !e; ++rep) {
            e = cudaEventRecord(e0, st);
            if (!e)
                rc = wrs_build_batched_rows_tuned(d_w, d_off, ntab, d_order, d_rows, d_ws, ws_bytes,
                                                  d_info, &x, stream);
            if (!e && !rc) e = cudaEventRecord(e1, st);
            if (!e && !rc) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (!e && !rc) e = cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 0 || ms < bestms) bestms = ms;
        }
        x.ms = bestms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc) return rc;
    if (e) return cuda_status(e);
    size_t bi = 0;
    for (size_t k = 1; k < cand.size(); ++k)
        if (cand[k].ms < cand[bi].ms) bi = k;
    // leave the buffers holding the chosen tiling's build (the same table)
    *best = cand[bi];
    if (all && nall) {
        const uint32_t m = (uint32_t)std::min<size_t>(*nall, cand.size());
        for (uint32_t k = 0; k < m; ++k) all[k] = cand[k];
    }
    if (nall) *nall = (uint32_t)cand.size();
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = *best;
    }
    return WRS_OK;
}

int wrs_sample_batched_rows(const wrs_row *d_rows, const uint64_t *d_off, uint32_t ntab,
                            const uint64_t *d_cnt_off, uint64_t seed, uint32_t *d_out,
                            void *stream) {
    if (ntab == 0) return WRS_OK;
    if (!d_rows || ((uintptr_t)d_rows & 7u) || !d_off || ((uintptr_t)d_off & 7u) || !d_cnt_off ||
        ((uintptr_t)d_cnt_off & 7u) || !d_out || ((uintptr_t)d_out & 3u))
        return WRS_EINVAL;
    return cuda_status(launch_sample_batched(d_rows, d_off, ntab, d_cnt_off, seed, d_out,
                                             (cudaStream_t)stream));
}

int wrs_diag_random_gather(const wrs_row *d_rows, uint64_t nrows, uint64_t count, uint64_t seed,
                           int flavor, uint32_t ctas_per_sm, uint32_t loads_in_flight,
                           uint32_t *d_out, void *stream) {
    if (!d_rows || nrows == 0 || ((uintptr_t)d_rows & 7u)) return WRS_EINVAL;
    if (count && (!d_out || ((uintptr_t)d_out & 3u))) return WRS_EINVAL;
    if (flavor < 0 || flavor > 2) return WRS_EINVAL;
    if (ctas_per_sm < 1 || ctas_per_sm > 64) return WRS_EINVAL;
    if (loads_in_flight != 4 && loads_in_flight != 8 && loads_in_flight != 16) return WRS_EINVAL;
    return cuda_status(launch_random_gather(d_rows, nrows, count, seed, flavor, ctas_per_sm,
                                            loads_in_flight, d_out, (cudaStream_t)stream));
}

int wrs_diag_pack_variant(const float *d_w, uint64_t n, wrs_row *d_rows, void *d_ws,
                          uint64_t ws_bytes, const wrs_config *cfg, uint32_t variant,
                          void *stream) {
    wrs_config c;
    Layout L;
    int rc = prep(n, d_ws, ws_bytes, cfg, &c, &L);
    if (rc) return rc;
    if (variant > 2 || !d_rows || ((uintptr_t)d_rows & 7u)) return WRS_EINVAL;
    if (variant == 0 && (!d_w || ((uintptr_t)d_w & 3u))) return WRS_EINVAL;
    return cuda_status(launch_pack_variant(d_w, n, d_rows, (unsigned char *)d_ws, L,
                                           c.section_size, variant, (cudaStream_t)stream));
}

int wrs_diag_prec_workspace_bytes(uint64_t n, const wrs_config *cfg, uint64_t *bytes) {
    wrs_config c;
    if (!bytes || n == 0 || n > kMaxN) return WRS_EINVAL;
    int rc = resolve_cfg(cfg, &c);
    if (rc) return rc;
    if (c.section_size > 1024) return WRS_EINVAL;
    *bytes = prec_workspace_bytes(n, c.section_size);
    return WRS_OK;
}

int wrs_diag_prec_split_pack(uint64_t n, wrs_row *d_rows, void *d_ws, uint64_t ws_bytes,
                             void *d_pws, uint64_t pws_bytes, const wrs_config *cfg,
                             uint32_t prec, void *stream) {
    wrs_config c;
    Layout L;
    int rc = prep(n, d_ws, ws_bytes, cfg, &c, &L);
    if (rc) return rc;
    if (prec > 1 || c.section_size > 1024 || !d_rows || ((uintptr_t)d_rows & 7u)) return WRS_EINVAL;
    if (!d_pws || ((uintptr_t)d_pws & 255u) || pws_bytes < prec_workspace_bytes(n, c.section_size))
        return WRS_EINVAL;
    return cuda_status(launch_prec_split_pack(n, d_rows, (unsigned char *)d_ws, L,
                                              (unsigned char *)d_pws, c.section_size, prec,
                                              (cudaStream_t)stream));
}

int wrs_diag_philox(uint64_t count, uint64_t seed, uint32_t *d_out, void *stream) {
    if (count && (!d_out || ((uintptr_t)d_out & 7u))) return WRS_EINVAL;
    return cuda_status(launch_philox_rate(count, seed, d_out, (cudaStream_t)stream));
}

}  // extern "C"
