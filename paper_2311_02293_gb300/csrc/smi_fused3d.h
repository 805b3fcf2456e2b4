// smi_fused3d.h -- the single-pass 3D step (smi_fused3d.cu): velocity and
// pressure updates of one leap-frog step with the CPML of all three axes
// inline, reading one buffer of the state and writing the other.
#pragma once

#include <cuda.h>

#include "smi_internal.h"

namespace smi {

// Tensor maps of one state buffer (p with its z- and x-widened tiles, the
// velocity components with theirs, the core tiles, and the full-size z / x
// CPML memory variables in the same geometries) ...
struct MapsF {
    CUtensorMap pA, pB, vzA, vxB, vy, pc, mzA, mxB, mzV, mxV;
};
// ... and of the model (rho widened along z and x, rho and kappa core tiles).
struct MapsM {
    CUtensorMap rA, rB, rc, Kc;
};

// True when the fused step can run: 3D, order 4 or 8, no free surface, a
// shot's field below 2^31 points, tensor-map encoder found.
bool fused3d_supported(const Grid &g);
bool make_maps_fused(MapsF &m, const Grid &g, const Fields &f, int nshot);
bool make_maps_model(MapsM &m, const Grid &g);

// One step (mode 0: forward at step `step`; 1: adjoint after `step` reverse
// steps) from state `cur` into state `nxt`.  The z and x CPML memory
// variables of both states are full-size arrays (ntot per shot), the y ones
// use the y-slab layout.  err: device word, bit 0 set if a bounded wait gave
// up.
void launch3_fused(const LaunchCtx &lc, const MapsF &mc, const MapsM &mm, const Grid &g, const Batch &b, Fields cur,
                   Fields nxt, int step, int mode, unsigned *err);

}  // namespace smi
