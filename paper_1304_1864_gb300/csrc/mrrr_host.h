// Host-side helpers shared by the entry points: the parameter defaults of a
// solve and the classification of caller pointers.
#pragma once

#include <cuda_runtime.h>

#include "mrrr.h"
#include "mrrr_types.cuh"

namespace mrrr {

// Paper defaults (Sec. 2, Sec. 3.2, Sec. 4.1); see mrrr.h for the fields.
//   gaptol: MIXED 1e-5 (x = binary32) / 1e-10 (x = binary64); PLAIN 3e-3 / 1e-3
//   xi:     MIXED 4 eps_x; PLAIN 8 eps_x ("Random perturbations", Sec. 3.2)
inline SolveCfg make_cfg(bool x_single, bool mixed, const mrrr_params* prm) {
    SolveCfg c;
    const double eps_s = 5.9604644775390625e-08, eps_d = 1.1102230246251565e-16, eps_dd = 4.930380657631324e-32;
    c.eps_x = x_single ? eps_s : eps_d;
    c.eps_y = mixed ? (x_single ? eps_d : eps_dd) : c.eps_x;
    c.mixed = mixed ? 1 : 0;
    double gt = mixed ? (x_single ? 1e-5 : 1e-10) : (x_single ? 3e-3 : 1e-3);
    double xi = mixed ? 4.0 * c.eps_x : 8.0 * c.eps_x;
    c.krs = 1.0;
    c.max_rqi = 10;
    c.seed = 0;
    c.flags = 0;
    if (prm) {
        if (prm->gaptol > 0) gt = prm->gaptol;
        if (prm->xi > 0) xi = prm->xi;
        if (prm->krs > 0) c.krs = prm->krs;
        if (prm->max_rqi > 0) c.max_rqi = prm->max_rqi;
        c.seed = prm->seed;
        c.flags = prm->flags;
    }
    c.gaptol = gt;
    c.rtol_class = 1e-2 * gt;
    c.xi = xi;
    c.growth_k = 8.0;
    return c;
}

// Where a caller's buffer lives.  Device (and managed) memory must belong to
// the device that is current at the call: a kernel of this device given
// another device's memory would access it without peer mapping.
enum PtrKind { PTR_HOST = 0, PTR_DEVICE = 1, PTR_OTHER_DEVICE = 2 };

inline PtrKind classify_ptr(const void* p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return PTR_HOST;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return PTR_HOST;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return PTR_OTHER_DEVICE;
    }
    // managed memory is reachable from every device; device memory only from its own
    if (a.type == cudaMemoryTypeDevice && a.device != cur) return PTR_OTHER_DEVICE;
    return PTR_DEVICE;
}

}  // namespace mrrr
