// xs_compute_noalloc: the line-sum cross-section for callers that cannot
// allocate device memory.
//
// Some callers of this library cannot call cudaMalloc (or any allocator) at the
// point where they need a cross-section: code running inside a host callback or
// a real-time loop that must not block on the driver's allocator, plugins
// hosted by a process whose memory pool is owned and capped by someone else,
// or tools that may only touch memory they were handed.  For them this entry
// point takes the scratch that xs_compute normally receives as a caller
// workspace from a fixed array compiled into the library instead.
//
// The array below is a file-scope __device__ variable: every GPU that loads
// libxs holds XS_NOALLOC_SCRATCH_BYTES of it until the process exits.  Host code
// may not use its name as an address (on the host it is only a shadow symbol),
// so the device address is looked up once per device with cudaGetSymbolAddress,
// with that device current, on the first call made on that device.
#include <mutex>

#include "xs_internal.h"

namespace {

constexpr size_t XS_NOALLOC_SCRATCH_BYTES = (size_t)64 << 20; // 64 MiB
constexpr int XS_NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[XS_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[XS_NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once).
int noalloc_scratch(void** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= XS_NOALLOC_MAX_DEVICES) return XS_ECUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return XS_ECUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return XS_OK;
}

} // namespace

extern "C" int xs_compute_noalloc(const xs_lines* lines, const double* nu, int64_t N, const double* T,
                                  const double* P_bar, int32_t L, double broad_scale, double wing_cut, int prec,
                                  void* sigma, xs_stream stream)
{
    XS_NVTX("xs_compute_noalloc");
    // the same argument checks as xs_compute
    int r = xsi::check_common(lines, nu, N, T, P_bar, L, broad_scale, wing_cut, prec);
    if (r) return r;
    if (!sigma) return XS_EINVAL;
    // the smallest plan (one layer at a time) must fit the fixed array
    if (xs_workspace_min_bytes(lines->n, N, L, prec) > XS_NOALLOC_SCRATCH_BYTES) return XS_ETOOBIG;
    void* scratch = nullptr;
    r = noalloc_scratch(&scratch);
    if (r != XS_OK) return r;
    // Every scratch region the forward pass reads is written earlier in the same
    // call (cut ranges, per-layer minima, line records, split-K partials), so the
    // previous call's contents never need clearing.
    return xsi::xs_run(lines, nu, N, T, P_bar, L, broad_scale, wing_cut, prec, sigma, scratch,
                       XS_NOALLOC_SCRATCH_BYTES, false, nullptr, nullptr, nullptr, (cudaStream_t)stream);
}
