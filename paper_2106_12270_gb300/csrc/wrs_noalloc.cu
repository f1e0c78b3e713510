// wrs_noalloc.cu - a build entry point that allocates nothing.
//
// Some callers cannot allocate device memory when they need a table: a
// service whose device memory plan is fixed at start-up (every byte is
// reserved up front and cudaMalloc afterwards is forbidden), or code running
// inside another framework that owns the allocator and whose accounting an
// extra cudaMalloc would break, or that must not suffer the implicit device
// synchronisation a cudaMalloc/cudaFree can bring.  wrs_build_rows already
// takes a caller workspace; this variant takes none at all: its workspace is
// a file-scope device array of a fixed size, kNoAllocBytes, which every GPU
// that loads this library holds until the process exits.
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
int cuda_status(cudaError_t e);
int resolve_cfg(const wrs_config *in, wrs_config *out);

constexpr uint64_t kNoAllocBytes = 32ull << 20;      // 32 MiB per GPU
constexpr uint64_t kNoAllocMaxItems = 3500000ull;    // a build's workspace fits in it

// The scratch.  In host code this name is only a host-side stand-in for the
// device array: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_ws[kNoAllocBytes];

// Device address of the scratch on the current device.  It is looked up on
// every call (the lookup allocates nothing and costs little), so a call made
// after the context was torn down and created again sees the array's new
// address.  The first lookup on a device loads this library's module there,
// which is why the first call on a device should come before any stream
// capture.
static cudaError_t noalloc_scratch(unsigned char **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_ws);
    if (e) return e;
    *out = static_cast<unsigned char *>(p);
    return cudaSuccess;
}

}  // namespace wrs

using namespace wrs;

extern "C" int wrs_build_rows_noalloc(const float *d_w, uint64_t n, wrs_row *d_rows,
                                      const wrs_config *cfg, wrs_build_info *d_info,
                                      void *stream) {
    wrs_config c;
    int rc = resolve_cfg(cfg, &c);
    if (rc) return rc;
    if (n == 0 || n > kNoAllocMaxItems) return WRS_EINVAL;
    if (!d_w || ((uintptr_t)d_w & 3u) || !d_rows || ((uintptr_t)d_rows & 7u) || !d_info)
        return WRS_EINVAL;
    Layout L = make_layout(n, c.section_size);
    if (L.total > kNoAllocBytes) return WRS_EINVAL;
    unsigned char *ws = nullptr;
    cudaError_t e = noalloc_scratch(&ws);
    cudaStream_t st = (cudaStream_t)stream;
    // every region the kernels read is written earlier in the same build (the
    // parameter block is cleared by launch_total), so whatever the previous
    // call left in the array does not matter
    if (!e) e = launch_total(d_w, n, ws, L, st);
    if (!e) e = launch_partition(d_w, n, ws, L, st);
    if (!e) e = launch_split(n, ws, L, c.section_size, c.split_method, st);
    if (!e) e = launch_pack(n, d_rows, ws, L, c.section_size, st);
    if (!e) e = launch_info(ws, L, d_info, st);
    return cuda_status(e);
}
