// md_apply_noalloc: the operator apply of md_apply with its scratch in a
// static device array instead of the operator's own buffers.
//
// Who needs it: callers that may not allocate device memory once they are
// running -- for example a solver embedded in a host application that
// reserves all device memory up front, or code that runs while another
// thread's allocator is forbidden to grow -- and callers that share one
// read-only operator handle between several users and so must not write the
// handle's scratch.  The call allocates nothing: the quadrature-point values
// t_q and a copy of the instance descriptor live in one file-scope
// __device__ array of MD_NOALLOC_BYTES bytes, which every GPU that loads the
// library holds until the process exits.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress and caches it for the life
// of the process (a cudaDeviceReset invalidates it); that first call should
// come before any stream capture.  All calls share the array and
// it keeps the last call's contents, so calls that overlap on the GPU (two
// streams, two threads) race with each other: order them.
#include <cstring>
#include <mutex>

#include "md_internal.h"

#define MD_NOALLOC_DESC_BYTES 1024
#define MD_NOALLOC_BYTES (MD_NOALLOC_DESC_BYTES + (size_t)MD_NOALLOC_MAX_NQ * sizeof(double))

// [instance descriptor (padded to 1 KB)][t_q, FP64 or FP32]
static __device__ __align__(256) unsigned char g_md_noalloc_scratch[MD_NOALLOC_BYTES];

static_assert(sizeof(InstDesc) <= MD_NOALLOC_DESC_BYTES, "descriptor does not fit its slot");

namespace {
std::mutex g_mu;
void* g_addr[64] = {};  // per device, the array's device address
}  // namespace

static md_status noalloc_base(void** out) {
    int dev = 0;
    MD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { md_set_error("md_apply_noalloc: device %d out of range", dev); return MD_ERR_ARG; }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_md_noalloc_scratch);
        if (e != cudaSuccess) return md_cuda_status(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return MD_OK;
}

// The descriptor is passed by value (a kernel parameter) and written into the
// array's descriptor slot on the caller's stream, so the call copies nothing
// from host memory.
__global__ void k_noalloc_desc(InstDesc d, InstDesc* dst) { *dst = d; }

extern "C" md_status md_apply_noalloc(const md_op* op, md_prec prec, const void* u, void* y, md_stream s) {
    if (!op || !u || !y) { md_set_error("md_apply_noalloc: NULL argument"); return MD_ERR_ARG; }
    if (prec != MD_FP32 && prec != MD_FP64) { md_set_error("md_apply_noalloc: bad precision"); return MD_ERR_ARG; }
    if (u == y) { md_set_error("md_apply_noalloc: u and y alias"); return MD_ERR_ARG; }
    if (op->h.nq > MD_NOALLOC_MAX_NQ) {
        md_set_error("md_apply_noalloc: %d quadrature points exceed the static scratch of %d", op->h.nq,
                     (int)MD_NOALLOC_MAX_NQ);
        return MD_ERR_ARG;
    }
    void* base = nullptr;
    MD_TRY(noalloc_base(&base));
    InstDesc d = op->h;
    unsigned char* t = static_cast<unsigned char*>(base) + MD_NOALLOC_DESC_BYTES;
    d.t64 = reinterpret_cast<double*>(t);
    d.t32 = reinterpret_cast<float*>(t);
    k_noalloc_desc<<<1, 1, 0, (cudaStream_t)s>>>(d, static_cast<InstDesc*>(base));
    MD_CHECK_LAUNCH();
    return launch_apply(op->tabs, static_cast<const InstDesc*>(base), 1, prec, u, op->off0, y, (cudaStream_t)s);
}
