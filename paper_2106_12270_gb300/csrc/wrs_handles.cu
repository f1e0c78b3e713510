// wrs_handles.cu - table and batch objects: the problem statement's interface
// (Sec. 1: build(weights) -> table, sample(table, count, seed) -> indices)
// over the buffer calls of wrs_api.cu.  A table owns its device rows; a
// build allocates its scratch in stream order and frees it when done.
#include <math.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "wrs_internal.cuh"

struct wrs_table {
    int device;
    uint64_t n;
    wrs_row *rows;      // device, owned (cudaMalloc)
    double W;
    uint64_t nl, nh;
};

struct wrs_batch {
    int device;
    uint32_t ntab;
    uint64_t total;
    wrs_row *rows;              // device, owned
    uint64_t *off;              // device copy of the offsets, owned
    wrs_table_summary *info;    // device, owned
};

namespace wrs {
int cuda_status(cudaError_t e);
int resolve_cfg(const wrs_config *in, wrs_config *out);
bool cached_batch_tuning(uint32_t ntab, uint64_t total, wrs_batch_tuning *out);

constexpr uint64_t kMaxItems = 0x7fffffffull;

std::mutex g_cfg_mu;
bool g_cfg_set = false;
wrs_config g_cfg;

static wrs_config current_config() {
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    wrs_config c;
    if (g_cfg_set) c = g_cfg;
    else wrs_config_default(&c);
    return c;
}

// Rows check of an imported table: prob in [0, 1] (not NaN) and alias < n;
// any violation sets *bad.
__global__ void k_check_rows(const wrs_row *__restrict__ rows, uint64_t n, uint32_t *bad) {
    uint32_t b = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const wrs_row r = rows[i];
        b |= !(r.prob >= 0.0f && r.prob <= 1.0f) || (uint64_t)r.alias >= n;
    }
    if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

extern int num_sms();

// Stream-ordered scratch of one call, freed on the same stream.
struct Scratch {
    void *p = nullptr;
    cudaStream_t st;
    explicit Scratch(cudaStream_t s) : st(s) {}
    cudaError_t alloc(uint64_t bytes) { return cudaMallocAsync(&p, bytes ? bytes : 1, st); }
    ~Scratch() {
        if (p) cudaFreeAsync(p, st);
    }
};

}  // namespace wrs

using namespace wrs;

extern "C" {

int wrs_set_config(const wrs_config *cfg) {
    wrs_config c;
    int rc = resolve_cfg(cfg, &c);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    g_cfg = c;
    g_cfg_set = true;
    return WRS_OK;
}

int wrs_get_config(wrs_config *cfg) {
    if (!cfg) return WRS_EINVAL;
    *cfg = current_config();
    return WRS_OK;
}

int wrs_build(const float *w, uint64_t n, int w_on_device, void *stream, wrs_table **out) {
    if (!out || !w || n == 0 || n > kMaxItems) return WRS_EINVAL;
    if (w_on_device && ((uintptr_t)w & 3u)) return WRS_EINVAL;
    const wrs_config c = current_config();
    uint64_t wsb = 0;
    int rc = wrs_build_workspace_bytes(n, &c, &wsb);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return cuda_status(e);
    wrs_table *t = new (std::nothrow) wrs_table();
    if (!t) return WRS_ENOMEM;
    t->device = dev;
    t->n = n;
    e = cudaMalloc(&t->rows, 8 * n);
    if (e) {
        delete t;
        return cuda_status(e);
    }
    // scratch: [build workspace][summary][weights copy, host input only]
    const uint64_t info_off = align_up(wsb, 256);
    const uint64_t w_off = info_off + align_up(sizeof(wrs_build_info), 256);
    const uint64_t total = w_off + (w_on_device ? 0 : 4 * n);
    wrs_build_info h_info;
    memset(&h_info, 0, sizeof h_info);
    {
        Scratch s(st);
        e = s.alloc(total);
        unsigned char *base = static_cast<unsigned char *>(s.p);
        const float *dw = w;
        if (!e && !w_on_device) {
            dw = reinterpret_cast<const float *>(base + w_off);
            e = cudaMemcpyAsync(const_cast<float *>(dw), w, 4 * n, cudaMemcpyHostToDevice, st);
        }
        wrs_build_info *d_info = reinterpret_cast<wrs_build_info *>(base + info_off);
        if (!e) {
            rc = wrs_build_rows(dw, n, t->rows, base, wsb, &c, d_info, stream);
            if (!rc) e = cudaMemcpyAsync(&h_info, d_info, sizeof h_info, cudaMemcpyDeviceToHost, st);
        }
    }   // scratch freed in stream order
    if (!e && !rc) e = cudaStreamSynchronize(st);
    if (!rc && e) rc = cuda_status(e);
    if (!rc) rc = h_info.status;
    if (rc) {
        cudaFree(t->rows);
        delete t;
        return rc;
    }
    t->W = h_info.W;
    t->nl = h_info.nl;
    t->nh = h_info.nh;
    *out = t;
    return WRS_OK;
}

int wrs_sample(const wrs_table *t, uint64_t count, uint64_t seed, uint32_t *d_out, int mode,
               void *stream) {
    if (!t || mode < WRS_SAMPLE_NAIVE || mode > WRS_SAMPLE_AUTO) return WRS_EINVAL;
    if (count && (!d_out || ((uintptr_t)d_out & 3u))) return WRS_EINVAL;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return cuda_status(e);
    if (dev != t->device) return WRS_EINVAL;
    if (count == 0) return WRS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (mode == WRS_SAMPLE_NAIVE)
        return wrs_sample_rows(t->rows, t->n, 0, count, seed, 0, WRS_TAG_NAIVE, d_out, stream);
    Scratch s(st);
    if (mode == WRS_SAMPLE_AUTO) {
        uint64_t b = 0;
        int rc = wrs_sample_auto_workspace_bytes(t->n, count, &b);
        if (rc) return rc;
        e = s.alloc(align_up(b, 256));
        if (e) return cuda_status(e);
        return wrs_sample_auto(t->rows, t->n, count, seed, d_out, s.p, align_up(b, 256), nullptr,
                               stream);
    }
    const uint32_t rows = mode == WRS_SAMPLE_SMEM ? 4096u : 8192u;
    uint64_t nsec = 0;
    int rc = wrs_sample_sections(t->n, rows, &nsec);
    if (rc) return rc;
    const uint64_t half = align_up(8 * nsec, 256);
    e = s.alloc(2 * half);
    if (e) return cuda_status(e);
    unsigned char *base = static_cast<unsigned char *>(s.p);
    return wrs_sample_sectioned_rows(t->rows, t->n, count, seed, (uint32_t)mode, rows,
                                     reinterpret_cast<uint64_t *>(base),
                                     reinterpret_cast<uint64_t *>(base + half), d_out, stream);
}

int wrs_table_info(const wrs_table *t, uint64_t *n, double *W, uint64_t *nl, uint64_t *nh) {
    if (!t) return WRS_EINVAL;
    if (n) *n = t->n;
    if (W) *W = t->W;
    if (nl) *nl = t->nl;
    if (nh) *nh = t->nh;
    return WRS_OK;
}

int wrs_table_rows(const wrs_table *t, const wrs_row **d_rows) {
    if (!t || !d_rows) return WRS_EINVAL;
    *d_rows = t->rows;
    return WRS_OK;
}

int wrs_table_export(const wrs_table *t, wrs_row *dst, int dst_on_device) {
    if (!t || !dst) return WRS_EINVAL;
    cudaError_t e = cudaMemcpy(dst, t->rows, 8 * t->n,
                               dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
    return cuda_status(e);
}

int wrs_table_import(const wrs_row *src, uint64_t n, int src_on_device, double W,
                     wrs_table **out) {
    if (!out || !src || n == 0 || n > kMaxItems) return WRS_EINVAL;
    if (src_on_device && ((uintptr_t)src & 7u)) return WRS_EINVAL;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return cuda_status(e);
    wrs_table *t = new (std::nothrow) wrs_table();
    if (!t) return WRS_ENOMEM;
    t->device = dev;
    t->n = n;
    t->W = W;
    t->nl = t->nh = UINT64_MAX;   // not known for an imported table
    uint32_t *d_bad = nullptr;
    uint32_t bad = 0;
    e = cudaMalloc(&t->rows, 8 * n);
    if (!e) e = cudaMemcpy(t->rows, src, 8 * n,
                           src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
    if (!e) e = cudaMalloc(&d_bad, sizeof(uint32_t));
    if (!e) e = cudaMemset(d_bad, 0, sizeof(uint32_t));
    if (!e) {
        const uint64_t want = (n + 255) / 256;
        const uint64_t cap = (uint64_t)num_sms() * 8;
        k_check_rows<<<(unsigned)(want < cap ? want : cap), 256>>>(t->rows, n, d_bad);
        e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpy(&bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost);
    if (d_bad) cudaFree(d_bad);
    int rc = e ? cuda_status(e) : (bad ? WRS_EINVAL : WRS_OK);
    if (rc) {
        if (t->rows) cudaFree(t->rows);
        delete t;
        return rc;
    }
    *out = t;
    return WRS_OK;
}

int wrs_table_destroy(wrs_table *t) {
    if (!t) return WRS_OK;
    int cur = 0;
    cudaError_t e = cudaGetDevice(&cur);
    if (!e && cur != t->device) e = cudaSetDevice(t->device);
    cudaError_t f = cudaFree(t->rows);
    if (!e && cur != t->device) cudaSetDevice(cur);
    delete t;
    return cuda_status(e ? e : f);
}

int wrs_build_batched(const float *d_w, const uint64_t *d_off, uint32_t ntab, void *stream,
                      wrs_batch **out) {
    if (!out || !d_w || ((uintptr_t)d_w & 3u) || !d_off || ((uintptr_t)d_off & 7u) || ntab == 0)
        return WRS_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return cuda_status(e);
    std::vector<uint64_t> h_off(ntab + 1);
    e = cudaMemcpyAsync(h_off.data(), d_off, 8 * (ntab + 1), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return cuda_status(e);
    if (h_off[0] != 0) return WRS_EINVAL;
    for (uint32_t k = 0; k < ntab; ++k)
        if (h_off[k + 1] < h_off[k]) return WRS_EINVAL;
    const uint64_t total = h_off[ntab];
    std::vector<uint32_t> order(ntab);
    int rc = wrs_batch_order(h_off.data(), ntab, order.data());
    if (rc) return rc;
    uint64_t wsb = 0;
    rc = wrs_build_batched_workspace_bytes(total, ntab, &wsb);
    if (rc) return rc;
    wrs_batch *b = new (std::nothrow) wrs_batch();
    if (!b) return WRS_ENOMEM;
    b->device = dev;
    b->ntab = ntab;
    b->total = total;
    e = cudaMalloc(&b->rows, 8 * (total ? total : 1));
    if (!e) e = cudaMalloc(&b->off, 8 * (uint64_t)(ntab + 1));
    if (!e) e = cudaMalloc(&b->info, sizeof(wrs_table_summary) * (uint64_t)ntab);
    if (!e) e = cudaMemcpyAsync(b->off, h_off.data(), 8 * (uint64_t)(ntab + 1),
                                cudaMemcpyHostToDevice, st);
    wrs_batch_tuning tune;
    const bool tuned = cached_batch_tuning(ntab, total, &tune);
    {
        Scratch s(st);
        const uint64_t ord_off = align_up(wsb, 256);
        if (!e) e = s.alloc(ord_off + 4 * (uint64_t)ntab);
        unsigned char *base = static_cast<unsigned char *>(s.p);
        uint32_t *d_order = reinterpret_cast<uint32_t *>(base + ord_off);
        if (!e) e = cudaMemcpyAsync(d_order, order.data(), 4 * (uint64_t)ntab,
                                    cudaMemcpyHostToDevice, st);
        if (!e)
            rc = wrs_build_batched_rows_tuned(d_w, b->off, ntab, d_order, b->rows, base, wsb,
                                              b->info, tuned ? &tune : nullptr, stream);
    }
    if (!e && !rc) e = cudaStreamSynchronize(st);   // host buffers above live until here
    if (!rc && e) rc = cuda_status(e);
    if (rc) {
        cudaFree(b->rows);
        cudaFree(b->off);
        cudaFree(b->info);
        delete b;
        return rc;
    }
    *out = b;
    return WRS_OK;
}

int wrs_batch_status(const wrs_batch *b, int32_t *h_status) {
    if (!b || !h_status) return WRS_EINVAL;
    std::vector<wrs_table_summary> s(b->ntab);
    cudaError_t e = cudaMemcpy(s.data(), b->info, sizeof(wrs_table_summary) * (uint64_t)b->ntab,
                               cudaMemcpyDeviceToHost);
    if (e) return cuda_status(e);
    for (uint32_t k = 0; k < b->ntab; ++k) h_status[k] = s[k].status;
    return WRS_OK;
}

int wrs_batch_summaries(const wrs_batch *b, wrs_table_summary *h_out) {
    if (!b || !h_out) return WRS_EINVAL;
    return cuda_status(cudaMemcpy(h_out, b->info, sizeof(wrs_table_summary) * (uint64_t)b->ntab,
                                  cudaMemcpyDeviceToHost));
}

int wrs_batch_rows(const wrs_batch *b, const wrs_row **d_rows, const uint64_t **d_off,
                   uint32_t *ntab) {
    if (!b) return WRS_EINVAL;
    if (d_rows) *d_rows = b->rows;
    if (d_off) *d_off = b->off;
    if (ntab) *ntab = b->ntab;
    return WRS_OK;
}

int wrs_batch_export(const wrs_batch *b, wrs_row *dst, int dst_on_device) {
    if (!b || !dst) return WRS_EINVAL;
    if (b->total == 0) return WRS_OK;
    return cuda_status(cudaMemcpy(dst, b->rows, 8 * b->total,
                                  dst_on_device ? cudaMemcpyDeviceToDevice
                                                : cudaMemcpyDeviceToHost));
}

int wrs_sample_batched(const wrs_batch *b, const uint64_t *d_cnt_off, uint64_t seed,
                       uint32_t *d_out, void *stream) {
    if (!b) return WRS_EINVAL;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return cuda_status(e);
    if (dev != b->device) return WRS_EINVAL;
    return wrs_sample_batched_rows(b->rows, b->off, b->ntab, d_cnt_off, seed, d_out, stream);
}

int wrs_batch_destroy(wrs_batch *b) {
    if (!b) return WRS_OK;
    int cur = 0;
    cudaError_t e = cudaGetDevice(&cur);
    if (!e && cur != b->device) e = cudaSetDevice(b->device);
    cudaError_t f = cudaFree(b->rows);
    cudaError_t g = cudaFree(b->off);
    cudaError_t h = cudaFree(b->info);
    if (!e && cur != b->device) cudaSetDevice(cur);
    delete b;
    return cuda_status(e ? e : f ? f : g ? g : h);
}

int wrs_diag_build_each(const float *d_w, const uint64_t *h_off, uint32_t ntab, wrs_row *d_rows,
                        void *d_ws, uint64_t ws_bytes, const wrs_config *cfg,
                        wrs_build_info *d_info, void *stream) {
    if (!h_off || (ntab && (!d_w || !d_rows || !d_info))) return WRS_EINVAL;
    for (uint32_t t = 0; t < ntab; ++t) {
        const uint64_t a = h_off[t], b = h_off[t + 1];
        if (b < a) return WRS_EINVAL;
        if (b == a) continue;
        int rc = wrs_build_rows(d_w + a, b - a, d_rows + a, d_ws, ws_bytes, cfg, d_info + t,
                                stream);
        if (rc) return rc;
    }
    return WRS_OK;
}

}  // extern "C"
