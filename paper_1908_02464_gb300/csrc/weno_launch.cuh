// Launch helpers: tile shapes per (dim, direction) and the host-side wrappers
// that pick a kernel instantiation.  Included by one translation unit per
// arithmetic (weno_f64.cu, weno_f32.cu, weno_mixed.cu) so that the three
// precisions compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "weno_adjoint.cuh"
#include "weno_kernels.cuh"
#include "weno_march.cuh"

namespace wis {

// Tile shapes: LINES grid lines of SEG cells along the sweep (plus a 3-cell
// halo on each side).  LINES x (SEG + 1) faces equal the CTA size, so the
// face phase runs in exactly one round (on the FP64 pipe a partly filled
// warp costs as much as a full one).  Variants:
//   0 long   2 x 63  halo work ~10%; y/z loads are 2-element row pieces
//   1 wide   8 x 15  8-element rows (coalesced y/z loads), halo work 40%
//   2 medium 4 x 31
// FP64 is ALU bound (variant 0 everywhere); FP32 y/z sweeps prefer coalesced
// rows.  weno_autotune times the variants on a live state and keeps the best.
//   3 single  1 x 127 halo work ~5%
//   4 small   1 x 95  96-thread CTAs (more resident CTAs per SM)
//   5 flat    123 consecutive faces of the line-after-line face sequence: no
//             partly filled tile at the end of each line (512 cells = 4 x 127
//             + 4 leaves a 4-cell tile per line otherwise), and a tile within
//             one line stages exactly 128 cells, one per thread, where 128
//             faces would leave a second round of 5 cells; lines shorter
//             than 122 cells take variant 3 instead
//   6 flat256 the flat tile with 251 faces on 256 threads (two CTAs per SM):
//             half the partly filled last warp per face, twice the WENO
//             faces per tile; lines shorter than 250 cells take variant 3
//   7 march   float y and z sweeps: k_march, one lane per line marching
//             along a segment (12 cells in 2D, 18 in 3D) with the stencil in
//             registers; float x sweeps take variant 3 and FP64 sweeps
//             variant 5 instead
constexpr int kTileVariants = 8;
template <int V> struct Tile;
template <> struct Tile<0> { static constexpr int LINES = 2, SEG = 63, NT = 128; static constexpr bool FLAT = false; };
template <> struct Tile<1> { static constexpr int LINES = 8, SEG = 15, NT = 128; static constexpr bool FLAT = false; };
template <> struct Tile<2> { static constexpr int LINES = 4, SEG = 31, NT = 128; static constexpr bool FLAT = false; };
template <> struct Tile<3> { static constexpr int LINES = 1, SEG = 127, NT = 128; static constexpr bool FLAT = false; };
template <> struct Tile<4> { static constexpr int LINES = 1, SEG = 95, NT = 96; static constexpr bool FLAT = false; };
template <> struct Tile<5> { static constexpr int LINES = 1, SEG = 122, NT = 128; static constexpr bool FLAT = true; };
template <> struct Tile<6> { static constexpr int LINES = 1, SEG = 250, NT = 256; static constexpr bool FLAT = true; };
struct Tile1D { static constexpr int LINES = 1, SEG = 127, NT = 128; static constexpr bool FLAT = false; };

template <typename T, int DIM, int DIR, bool EXACTDET, typename TL>
cudaError_t launch_sweep_one(const SweepArgs& a, cudaStream_t s)
{
    using SM = SweepSmem<T, DIM, TL::LINES, TL::SEG, TL::FLAT>;
    auto kern = k_sweep<T, DIM, DIR, TL::LINES, TL::SEG, TL::NT, EXACTDET, TL::FLAT>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int nd = a.n[DIR];
    const int segs = (nd + TL::SEG - 1) / TL::SEG;
    dim3 grid;
    if (TL::FLAT) {
        // tile t holds faces t SEG .. t SEG + SEG of the (nd + 1) x lines face sequence
        const long long lines = DIR == 0 ? (long long)a.n[1] * a.n[2]
                                         : (DIR == 1 ? (long long)a.n[0] * a.n[2] : (long long)a.n[0] * a.n[1]);
        const long long faces = (long long)(nd + 1) * lines;
        grid = dim3((unsigned)((faces - 1 + TL::SEG - 1) / TL::SEG));
    } else if (DIR == 0) grid = dim3(segs, (a.n[1] + TL::LINES - 1) / TL::LINES, a.n[2]);
    else if (DIR == 1) grid = dim3((a.n[0] + TL::LINES - 1) / TL::LINES, segs, a.n[2]);
    else grid = dim3((a.n[0] + TL::LINES - 1) / TL::LINES, a.n[1], segs);
    return launch_pdl(kern, grid, dim3(TL::NT), SM::bytes, s, a);
}

template <typename T, int DIM, int DIR, bool EXACTDET>
cudaError_t launch_sweep_v(int variant, const SweepArgs& a, cudaStream_t s)
{
    if (variant == 1) return launch_sweep_one<T, DIM, DIR, EXACTDET, Tile<1>>(a, s);
    if (variant == 2) return launch_sweep_one<T, DIM, DIR, EXACTDET, Tile<2>>(a, s);
    if (variant == 3) return launch_sweep_one<T, DIM, DIR, EXACTDET, Tile<3>>(a, s);
    if (variant == 4) return launch_sweep_one<T, DIM, DIR, EXACTDET, Tile<4>>(a, s);
    if (variant == 5) {
        if (a.n[DIR] >= Tile<5>::SEG) return launch_sweep_one<T, DIM, DIR, EXACTDET, Tile<5>>(a, s);
        return launch_sweep_one<T, DIM, DIR, EXACTDET, Tile<3>>(a, s);
    }
    if (variant == 6) {
        if (a.n[DIR] >= Tile<6>::SEG) return launch_sweep_one<T, DIM, DIR, EXACTDET, Tile<6>>(a, s);
        return launch_sweep_one<T, DIM, DIR, EXACTDET, Tile<3>>(a, s);
    }
    if (variant == 7) {
        if constexpr (sizeof(T) == 4 && DIR >= 1) {
            if (a.P == nullptr && a.Pout == nullptr) return launch_march<T, DIM, DIR, EXACTDET>(a, s);
        }
        if (sizeof(T) == 4) return launch_sweep_one<T, DIM, DIR, EXACTDET, Tile<3>>(a, s);
        return launch_sweep_v<T, DIM, DIR, EXACTDET>(5, a, s);
    }
    return launch_sweep_one<T, DIM, DIR, EXACTDET, Tile<0>>(a, s);
}

template <typename T, bool EXACTDET>
cudaError_t launch_sweep_t(int dim, int dir, int variant, const SweepArgs& a, cudaStream_t s)
{
    if (dim == 1) return launch_sweep_one<T, 1, 0, EXACTDET, Tile1D>(a, s);
    if (dim == 2) {
        if (dir == 0) return launch_sweep_v<T, 2, 0, EXACTDET>(variant, a, s);
        return launch_sweep_v<T, 2, 1, EXACTDET>(variant, a, s);
    }
    if (dir == 0) return launch_sweep_v<T, 3, 0, EXACTDET>(variant, a, s);
    if (dir == 1) return launch_sweep_v<T, 3, 1, EXACTDET>(variant, a, s);
    return launch_sweep_v<T, 3, 2, EXACTDET>(variant, a, s);
}

inline int grid_for(long long work, int threads, int cap)
{
    long long b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

template <typename T>
cudaError_t launch_cfl_t(int dim, const CflArgs& a_in, int nsm, cudaStream_t s)
{
    // rows x parts units of at least 256 cells each, about 8 blocks per SM
    CflArgs a = a_in;
    const long long rows = (long long)a.n[1] * a.n[2];
    const long long want = (long long)nsm * 8;
    long long parts = (want + rows - 1) / rows;
    const long long most = (a.n[0] + 255) / 256;
    if (parts > most) parts = most;
    if (parts < 1) parts = 1;
    a.parts = (int)parts;
    const int blocks = grid_for(rows * parts * 256, 256, nsm * 8);
    if (dim == 1) return launch_pdl(k_cfl<T, 1>, dim3(blocks), dim3(256), 0, s, a);
    if (dim == 2) return launch_pdl(k_cfl<T, 2>, dim3(blocks), dim3(256), 0, s, a);
    return launch_pdl(k_cfl<T, 3>, dim3(blocks), dim3(256), 0, s, a);
}

template <typename T>
cudaError_t launch_lf_t(int dim, const CflArgs& a, unsigned long long* out, int nsm, cudaStream_t s)
{
    const long long cells = (long long)a.n[0] * a.n[1] * a.n[2];
    const int blocks = grid_for(cells, 256, nsm * 8);
    if (dim == 1) return launch_pdl(k_lf_alpha<T, 1>, dim3(blocks), dim3(256), 0, s, a, out);
    if (dim == 2) return launch_pdl(k_lf_alpha<T, 2>, dim3(blocks), dim3(256), 0, s, a, out);
    return launch_pdl(k_lf_alpha<T, 3>, dim3(blocks), dim3(256), 0, s, a, out);
}

template <typename T>
cudaError_t launch_totals_t(int dim, const TotArgs& a, int blocks, cudaStream_t s)
{
    if (dim == 1) k_totals<T, 1><<<blocks, 256, 0, s>>>(a);
    else if (dim == 2) k_totals<T, 2><<<blocks, 256, 0, s>>>(a);
    else k_totals<T, 3><<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pack_t(const void* src, void* dst, int nv, const int* n, long long sy, long long sz,
                          long long sv, long long off0, int to_ghosted, int nsm, cudaStream_t s)
{
    // units of 256 consecutive cells of one row (see k_pack)
    const long long units = (long long)nv * n[1] * n[2] * ((n[0] + 255) / 256);
    const int blocks = (int)(units < (long long)nsm * 16 ? units : (long long)nsm * 16);
    k_pack<T><<<blocks, 256, 0, s>>>(reinterpret_cast<const T*>(src), reinterpret_cast<T*>(dst), nv, n[0],
                                      n[1], n[2], sy, sz, sv, off0, to_ghosted);
    return cudaGetLastError();
}

// grid of the adjoint tiles of one direction (both passes use it)
template <typename T, int DIM, int DIR>
dim3 vjp_grid(const int* n)
{
    using TL = VjpTile<T, DIM, DIR>;
    int e0, e1;
    // y and z tiles hold TL::LINES lines consecutive in x
    if (DIR == 0) { e0 = n[1]; e1 = n[2]; }
    else if (DIR == 1) { e0 = (n[0] + TL::LINES - 1) / TL::LINES; e1 = n[2]; }
    else { e0 = (n[0] + TL::LINES - 1) / TL::LINES; e1 = n[1]; }
    return dim3((n[DIR] + TL::SEG - 1) / TL::SEG, e0, e1);
}

template <typename T, int DIM, int DIR, int PASS>
cudaError_t launch_vjp_pass(const VjpArgs& a, cudaStream_t s)
{
    using SM = VjpSmem<T, DIM, DIR, PASS>;
    constexpr int NT = VjpTile<T, DIM, DIR>::NT;
    auto kern = k_vjp<T, DIM, DIR, PASS>;
    static int resident = 0;   // CTAs per SM (pass 1 grid)
    if (resident == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kern, NT, SM::bytes);
        if (e != cudaSuccess) return e;
        if (resident < 1) resident = 1;
    }
    const dim3 g = vjp_grid<T, DIM, DIR>(a.n);
    VjpArgs b = a;
    b.tiles[0] = (int)g.x; b.tiles[1] = (int)g.y; b.tiles[2] = (int)g.z;
    if (PASS == 0) {
        kern<<<g, NT, SM::bytes, s>>>(b);
    } else {
        int dev = 0, nsm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const long long tiles = (long long)g.x * g.y * g.z;
        const long long blocks = (long long)resident * nsm < tiles ? (long long)resident * nsm : tiles;
        kern<<<(unsigned)(blocks > 0 ? blocks : 1), NT, SM::bytes, s>>>(b);
    }
    return cudaGetLastError();
}

// pass 0 (linear-upwind faces, lists the tiles with WENO faces), then pass 1
// (the WENO faces of the listed tiles)
template <typename T, int DIM, int DIR>
cudaError_t launch_vjp_one(const VjpArgs& a, cudaStream_t s)
{
    cudaError_t e = launch_vjp_pass<T, DIM, DIR, 0>(a, s);
    if (e != cudaSuccess) return e;
    return launch_vjp_pass<T, DIM, DIR, 1>(a, s);
}

template <typename T>
cudaError_t launch_vjp_t(int dim, int dir, const VjpArgs& a, cudaStream_t s)
{
    if (dim == 1) return launch_vjp_one<T, 1, 0>(a, s);
    if (dim == 2) return dir == 0 ? launch_vjp_one<T, 2, 0>(a, s) : launch_vjp_one<T, 2, 1>(a, s);
    if (dir == 0) return launch_vjp_one<T, 3, 0>(a, s);
    if (dir == 1) return launch_vjp_one<T, 3, 1>(a, s);
    return launch_vjp_one<T, 3, 2>(a, s);
}

// number of adjoint tiles of one direction (the most VjpArgs::weno_tiles holds)
template <typename T>
long long vjp_tiles_t(int dim, int dir, const int* n)
{
    dim3 g;
    if (dim == 1) g = vjp_grid<T, 1, 0>(n);
    else if (dim == 2) g = dir == 0 ? vjp_grid<T, 2, 0>(n) : vjp_grid<T, 2, 1>(n);
    else g = dir == 0 ? vjp_grid<T, 3, 0>(n) : (dir == 1 ? vjp_grid<T, 3, 1>(n) : vjp_grid<T, 3, 2>(n));
    return (long long)g.x * g.y * g.z;
}

template <typename T>
cudaError_t launch_ghost_adj_t(int dim, const GhostArgs& a, const void* ghost, void* G, cudaStream_t s)
{
    long long P;
    if (a.dir == 0) P = (long long)a.n[1] * a.n[2];
    else if (a.dir == 1) P = (long long)a.n[0] * a.n[2];
    else P = (long long)a.n[0] * a.n[1];
    const int blocks = grid_for(P, 256, 4096);
    if (dim == 1) k_ghost_adj<T, 1><<<blocks, 256, 0, s>>>(a, ghost, G);
    else if (dim == 2) k_ghost_adj<T, 2><<<blocks, 256, 0, s>>>(a, ghost, G);
    else k_ghost_adj<T, 3><<<blocks, 256, 0, s>>>(a, ghost, G);
    return cudaGetLastError();
}

// per-precision entry points (one translation unit each)
cudaError_t vjp_f64(int dim, int dir, const VjpArgs& a, cudaStream_t s);
cudaError_t vjp_f32(int dim, int dir, const VjpArgs& a, cudaStream_t s);
long long vjp_tiles_f64(int dim, int dir, const int* n);
long long vjp_tiles_f32(int dim, int dir, const int* n);
cudaError_t ghost_adj_f64(int dim, const GhostArgs& a, const void* ghost, void* G, cudaStream_t s);
cudaError_t ghost_adj_f32(int dim, const GhostArgs& a, const void* ghost, void* G, cudaStream_t s);
cudaError_t sweep_f64(int dim, int dir, int variant, const SweepArgs& a, cudaStream_t s);
cudaError_t sweep_f32(int dim, int dir, int variant, const SweepArgs& a, cudaStream_t s);
cudaError_t sweep_mixed(int dim, int dir, int variant, const SweepArgs& a, cudaStream_t s);
cudaError_t cfl_f64(int dim, const CflArgs& a, int nsm, cudaStream_t s);
cudaError_t cfl_f32(int dim, const CflArgs& a, int nsm, cudaStream_t s);
cudaError_t lf_f64(int dim, const CflArgs& a, unsigned long long* out, int nsm, cudaStream_t s);
cudaError_t lf_f32(int dim, const CflArgs& a, unsigned long long* out, int nsm, cudaStream_t s);
cudaError_t totals_f64(int dim, const TotArgs& a, int blocks, cudaStream_t s);
cudaError_t totals_f32(int dim, const TotArgs& a, int blocks, cudaStream_t s);
cudaError_t pack_f64(const void* src, void* dst, int nv, const int* n, long long sy, long long sz, long long sv,
                     long long off0, int to_ghosted, int nsm, cudaStream_t s);
cudaError_t pack_f32(const void* src, void* dst, int nv, const int* n, long long sy, long long sz, long long sv,
                     long long off0, int to_ghosted, int nsm, cudaStream_t s);

}  // namespace wis
