// Error reporting and version of the md library.
#include <cstdarg>
#include <cstdio>

#include "md_internal.h"

namespace {
thread_local char g_err[1024] = "";
}

void md_set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

md_status md_cuda_status(cudaError_t e, const char* what, const char* file, int line) {
    md_set_error("%s failed at %s:%d: %s", what, file, line, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return MD_ERR_OOM;
    return MD_ERR_CUDA;
}

extern "C" const char* md_last_error(void) { return g_err; }
extern "C" const char* md_version(void) { return "md-gb300 0.1 (sm_103a)"; }
