// Launch configuration of the fused step kernel: tile shape, ring depths and
// the z-chunk decomposition.  Everything that decides the kernel's memory
// traffic lives here and in step_kernel.cuh.
#pragma once
#include <cuda.h>

#include "step_kernel.cuh"

namespace sgb {

// Tile configuration (build-time): threads in x (4 points each), threads in y,
// rows per thread, u-ring stages, (u^{n-1}, m, phi)-ring stages, min CTAs/SM.
#ifndef SGB_TXT
#define SGB_TXT 16
#endif
#ifndef SGB_TYT
#define SGB_TYT 8
#endif
#ifndef SGB_TY
#define SGB_TY 2
#endif
#ifndef SGB_UNROLL
#define SGB_UNROLL 1
#endif
#ifndef SGB_NU
#define SGB_NU 9
#endif
#ifndef SGB_NP
#define SGB_NP 4
#endif
#ifndef SGB_MINB
#define SGB_MINB 2
#endif
// L2 promotion of the tensor maps: the u^n box with its x-y halo (the
// halos are shared with neighbouring tiles, so wider L2 fills are reused),
// and the halo-free tiles (u^{n-1}, m, phi, ...), whose rows are whole 32-byte
// sectors that no other tile reads: promoting those fetched sectors nobody
// used (measured on 256^3 + 16-point PML: 14 MB less DRAM read per step
// without promotion, 2% faster on 512^3).
#ifndef SGB_L2PROMO
#define SGB_L2PROMO CU_TENSOR_MAP_L2_PROMOTION_L2_256B
#endif
#ifndef SGB_L2PROMO_P
#define SGB_L2PROMO_P CU_TENSOR_MAP_L2_PROMOTION_NONE
#endif
using Cfg = TileCfg<SGB_TXT, SGB_TYT, SGB_TY, SGB_NU, SGB_NP, SGB_MINB, SGB_UNROLL>;

// Chunking of z: pick the chunk length that minimises waves x (chunk + priming
// overhead) for the resident-CTA slots of this GPU.  Chunks are capped at 40
// planes: CTAs of tiles in the x-y PML band move 1.5x the bytes per plane of
// interior tiles, so neighbours drift apart in z over long chunks and their
// shared halos fall out of L2 (measured on 512^3: 22-40-plane chunks move ~10%
// fewer DRAM bytes than 74-plane chunks; with the 9-stage u^n ring 40-plane
// chunks ran 1.7% faster than 27-plane ones, 52- and 64-plane chunks slower).
inline void choose_decomposition(int Nx, int Ny, int Nz, int sms, int occ, StepArgs &a, int *grid)
{
    a.tiles_x = (Nx + Cfg::BX - 1) / Cfg::BX;
    a.tiles_y = (Ny + Cfg::BY - 1) / Cfg::BY;
    const long long tiles = (long long)a.tiles_x * a.tiles_y;
    const long long slots = (long long)sms * occ;
    int best_zc = Nz;
    double best = 1e300;
#ifdef SGB_FORCE_CHUNKS
    {
        const int zc = (Nz + SGB_FORCE_CHUNKS - 1) / SGB_FORCE_CHUNKS;
        a.zc = zc;
        *grid = (int)(tiles * ((Nz + zc - 1) / zc));
        return;
    }
#endif
    const int cmax = Nz / 4 > 1 ? Nz / 4 : 1;
    for (int c = 1; c <= cmax; ++c) {
        const int zc = (Nz + c - 1) / c;
        if (zc > 40 && c < cmax) continue;
        const int ceff = (Nz + zc - 1) / zc;
        const long long units = tiles * ceff;
        const long long waves = (units + slots - 1) / slots;
        const double cost = (double)waves * (zc + 8 * 0.5);
        if (cost < best * 0.999) {
            best = cost;
            best_zc = zc;
        }
    }
    a.zc = best_zc;
    *grid = (int)(tiles * ((Nz + best_zc - 1) / best_zc));
}


}  // namespace sgb
