// Error reporting and library metadata.
#include <stdio.h>

#include <string>

#include "gj_internal.h"

namespace gj {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

gj_status cuda_fail(cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    set_error(m);
    return e == cudaErrorMemoryAllocation ? GJ_ERR_OOM : GJ_ERR_CUDA;
}

}  // namespace gj

extern "C" const char *gj_last_error(void) { return gj::g_last_error.c_str(); }

extern "C" const char *gj_version(void) { return "gj 0.1 (sm_103a)"; }
