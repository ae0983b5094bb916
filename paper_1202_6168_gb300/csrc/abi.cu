// abi.cu - error reporting, version and option defaults of the C ABI.
#include <cstdarg>

#include "di_internal.cuh"

namespace di {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

}  // namespace di

extern "C" DI_API const char *di_version(void) { return "di-gb300 0.1.0 (sm_103a)"; }

extern "C" DI_API const char *di_last_error(void) { return di::g_err; }

extern "C" DI_API di_status di_opts_default(di_opts *o) {
    if (!o) {
        di::set_error("di_opts_default: NULL");
        return DI_EINVAL;
    }
    std::memset(o, 0, sizeof(*o));
    o->alpha = 1.5;
    o->fluid_fp64 = 0;
    o->recompute_every = 0;
    o->recompute_drop = 1024.0;
    o->max_levels = 100000;
    o->warm_start = 0;
    o->warm_fallback = 1;
    o->l2_window = 1;
    o->timing = 0;
    o->propagation = 3;
    o->push_ratio = 8;
    o->exact_residual = 0;
    o->selection = 0;
    o->dangling = 0;
    o->spin_limit = 1LL << 20;
    o->stream = nullptr;
    o->resweeps = 0;
    o->slice_sweeps = -1;
    return DI_OK;
}
