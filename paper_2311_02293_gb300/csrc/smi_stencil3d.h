// smi_stencil3d.h -- TMA-streamed 3D stencil kernels (smi_stencil3d.cu).
#pragma once

#include <cuda.h>

#include "smi_internal.h"

namespace smi {

// Tensor maps of one batch's fields (haloed plane tiles and 32 x 16 core
// tiles) and of the model arrays.
struct Maps3 {
    CUtensorMap p_halo, p_core, vz_core, vx_core, vy_core, vz_halo, vx_halo, rho_v, K_core;
    // full-size z / x CPML memory variables (inline band terms): the p-grid ones
    // (psiv) in the p tile geometry and core, the v-grid ones (psip) core and in
    // the v_z / v_x tile geometries
    CUtensorMap pz_halo, px_halo, pz_core, px_core, cz_core, cx_core, cz_vhalo, cx_vhalo;
};

// One warp waits with the tile kernels' bounded-wait helper on an mbarrier
// that nothing completes, for `polls` polls, then sets bit 0 of err.
void launch_wait_check(const LaunchCtx &lc, unsigned *err, long long polls);
// The polls after which a tile kernel's wait gives up.
long long wait_polls_default();

// 4D tensor map (z, x, y, shot) over nshot padded fields starting at base,
// with a box of bz (z) x bx (x) x 1 x 1 and zero fill out of bounds; false if
// the encoder is missing or refuses the map.
bool make_tile_map(CUtensorMap *tm, const Grid &g, const float *base, int nshot, int bz, int bx);

// True when the 3D kernels can run (3D, order 4 or 8, tensor-map encoder found).
bool stencil3d_supported(const Grid &g);

// Builds the maps for fields f of a batch of nshot shots (fullmem: the z / x
// memory variables are full-size arrays, whose maps the inline band terms
// read); false on failure.
bool make_maps3(Maps3 &m, const Grid &g, const Fields &f, int nshot, bool fullmem);

// mode 0: forward, 1: adjoint (step = reverse steps elapsed), 2: reconstruction.
// err: device word, bit 0 set if a bounded wait gave up.
// inl (modes 0 and 1): the z / x CPML terms inline (interior and band tile
// classes; full-size memory variables); else they are left to the band
// kernels (launch_fwd_corrections / launch_adj_corrections).
void launch3_v(const LaunchCtx &lc, const Maps3 &m, const Grid &g, const Batch &b, Fields f, int step, int mode,
               unsigned *err, bool inl);
// lpm: maps of the adjoint fields, whose pressure the reconstruction mode
// correlates with (mode 2 only).
void launch3_p(const LaunchCtx &lc, const Maps3 &m, const Maps3 *lpm, const Grid &g, const Batch &b, Fields f,
               int step, int mode, unsigned *err, float *acc, int img_mode, const float *stf, float src_scale, bool inl);

}  // namespace smi
