// Kernels of the regularized WENO-IS Euler solver (sm_103a).
//
//   k_sweep   one direction of the semi-discrete operator (Eq. goveq5): a
//             tile of LINES grid lines x SEG cells along the sweep (or 123
//             consecutive faces of the line-after-line face sequence),
//             staged in shared memory with a 3-cell halo whose ghost cells
//             come from the boundary conditions; every face of the tile goes
//             through the detector (Eq. eq27-28) and either the optimal
//             linear upwind flux (Eq. linearupwind) or, after compaction
//             into a per-tile queue, the characteristic regularized WENO-IS
//             flux (Sec. 2.4, Eq. eq8-r); the tile then takes the flux
//             divergence and writes an accumulator, a right-hand side or the
//             RK3 stage combination (Sec. 4).
//   k_cfl     CFL wave-speed max-reduction and admissibility check.
//   k_dt, k_post   single-thread time-step bookkeeping on the device.
//   k_totals  conserved totals, FP64 accumulation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "weno_device.cuh"

namespace wis {

// Programmatic dependent launch.  The kernels of a time step are launched
// with programmatic stream serialization (launch_pdl), so that a kernel's
// CTAs can become resident while its predecessor's last wave finishes.
// Every such kernel calls pdl_enter before its first access to global
// memory: griddepcontrol.wait returns once the predecessor grid has
// completed and its writes are visible (at once for an ordinary launch),
// and launch_dependents then lets the successor launch.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              A&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}

// Device-resident time state of a context.
struct DevTime {
    double t;                       // time of the current state
    double dt;                      // step in progress (0: nothing to do)
    double t_end;                   // target of the step in progress
    unsigned long long smax_bits;   // max wave speed sum (bits of a positive double)
    long long steps;                // completed steps
    int status;                     // 0 ok, else WENO_ERR_NONPHYSICAL latched
    int clipped;                    // 1 if dt was clipped to reach t_end
    double xs_top[3];               // double Mach top boundary: shock position at the
                                    // stage times t, t + dt, t + dt/2
};

// Shock position on the top boundary of the double Mach reflection at time t
// (the Mach 10 shock through (1/6, 0) at 60 degrees moves at 10 / sin 60).
__host__ __device__ inline double dmr_shock_x(double t) { return 1.0 / 6.0 + (1.0 + 20.0 * t) / sqrt(3.0); }

enum { MODE_ACC_SET = 0, MODE_ACC_ADD = 1, MODE_COMBINE = 2, MODE_RHS = 3 };
// flux splitting (Eq. flxuspliting): local LF over the six stencil cells,
// global LF over the domain, Roe (the Roe-average eigenvalue)
enum { SPLIT_LLF = 0, SPLIT_LF = 1, SPLIT_RF = 2 };

struct SweepArgs {
    const void* U;      // stage input, ghosted layout
    const void* Un;     // RK base state (COMBINE with rk_a != 0), ghosted
    void* acc;          // accumulated RHS of earlier directions (may be null)
    void* out;          // COMBINE: next stage state; RHS: right-hand side
    int mode;
    double rk_a, rk_b;  // out = rk_a Un + rk_b (U + dt rhs)
    DevTime* tm;        // null for a stand-alone RHS evaluation
    unsigned long long* weno_count;
    uint8_t* flags;     // per-face flags of this direction (may be null)
    int n[3];
    long long sy, sz, sv, off0;
    double inv_dx, eps_h, gamma, eps, c_lambda;
    double slim;                    // 60 sqrt(eps_h): the detector threshold on |60 dv^s| / rho~
    int hybrid;
    int wmode;                      // W_REG, W_IS, W_WANG, W_LINEAR
    int split;                      // SPLIT_LLF, SPLIT_LF, SPLIT_RF
    const unsigned long long* alpha_g;  // SPLIT_LF: bits of max |u-c|, |u|, |u+c| of this direction
    // the same constants pre-rounded for float kernels (a double conversion
    // or division per thread would run on the slow FP64 pipe)
    float inv_dx_f, gamma_f, eps_f, slim_f, lam_scale_f, rk_a_f, rk_b_f;
    // boundary conditions of this direction, applied while staging the tile
    // (the ghost cells are computed, not read)
    int bc_lo, bc_hi;
    double bc_state[2][5];
    float bc_state_f[2][5];
    double lo0, dx0, lo1, dx1;   // x and y geometry (double Mach, jet)
    int stage;                   // RK stage (index of tm->xs_top)
    double xs_fixed;             // double Mach shock position when tm is null
    // Primitives (cell_prims) of U's interior cells: the record of the cell
    // at index g of U's layout at P + PrimLayout::STRIDE g.  P: read them (the first sweep of the stage
    // wrote them); Pout: the tiles compute them and store those of their own
    // cells; both null: the tiles compute them and keep them to themselves.
    const void* P = nullptr;
    void* Pout = nullptr;
    // Scale of the accumulator `acc` as this sweep reads it (ACC_ADD, RHS,
    // COMBINE): MODE_ACC_SET stores the plain difference of the (times 60)
    // face fluxes, so its reader multiplies by that direction's 1/(60 dx);
    // an ACC_ADD accumulator is already scaled (1).
    double acc_scale = 1.0;
    float acc_scale_f = 1.0f;
};

template <typename T> __device__ __forceinline__ T pick(double d, float f);
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }

enum { BC_TRANSMISSIVE = 0, BC_REFLECT = 1, BC_PERIODIC = 2, BC_INFLOW = 3, BC_DMR_BOTTOM = 4,
       BC_DMR_TOP = 5, BC_JET = 6 };

// half width of the inflow jet (bc_state[0] where y < JET_HALF_WIDTH)
constexpr double JET_HALF_WIDTH = 0.05;

// Where the state of cell `along` of a grid line comes from (interior or
// one of the three ghost cells per side), applying the boundary condition of
// direction DIR: transmissive (nearest interior cell), reflecting (mirror,
// normal momentum negated), periodic (wrap), fixed states (inflow, double
// Mach bottom and top, jet).  `line` indexes the grid line: the row j for x
// sweeps, the column i for y/z sweeps.  Returns the fixed state's index
// (0 or 1) or -1 with the source cell's global index in g and whether its
// normal momentum is negated in flip.
template <int DIR>
__device__ __forceinline__ int cell_source(const SweepArgs& a, long long line_base, int line, int along, int nd,
                                           long long& g, bool& flip)
{
    const long long sd = DIR == 0 ? 1LL : (DIR == 1 ? a.sy : a.sz);
    int src = along;
    flip = false;
    if (along < 0 || along >= nd) {
        const int side = along < 0 ? 0 : 1;
        const int gl = side == 0 ? -along : along - nd + 1;
        int bc = side == 0 ? a.bc_lo : a.bc_hi;
        int fixed = -1;
        if (bc == BC_INFLOW) {
            fixed = 0;
        } else if (bc == BC_DMR_BOTTOM) {
            const double x = a.lo0 + (line + 0.5) * a.dx0;
            if (x < 1.0 / 6.0) fixed = 0;
            else bc = BC_REFLECT;
        } else if (bc == BC_DMR_TOP) {
            // shock position on the top boundary at the boundary time
            const double xs = a.tm != nullptr ? a.tm->xs_top[a.stage] : a.xs_fixed;
            const double x = a.lo0 + (line + 0.5) * a.dx0;
            fixed = x < xs ? 0 : 1;
        } else if (bc == BC_JET) {
            const double y = a.lo1 + (line + 0.5) * a.dx1;
            fixed = y < JET_HALF_WIDTH ? 0 : 1;
        }
        if (fixed >= 0) return fixed;
        if (bc == BC_TRANSMISSIVE) src = side == 0 ? 0 : nd - 1;
        else if (bc == BC_REFLECT) { src = side == 0 ? gl - 1 : nd - gl; flip = true; }
        else src = side == 0 ? nd - gl : gl - 1;
    }
    g = line_base + (long long)src * sd;
    return -1;
}

// State of cell `along` of a grid line (see cell_source).
template <typename T, int DIM, int DIR>
__device__ __forceinline__ void stage_cell(const SweepArgs& a, const T* Ug, long long line_base, int line, int along,
                                           int nd, T* U)
{
    constexpr int NV = DIM + 2;
    long long g = 0;
    bool flip = false;
    const int fixed = cell_source<DIR>(a, line_base, line, along, nd, g, flip);
    if (fixed >= 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = pick<T>(a.bc_state[fixed][v], a.bc_state_f[fixed][v]);
        return;
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) U[v] = Ug[g + v * a.sv];
    if (flip) U[1 + DIR] = -U[1 + DIR];
}

// Cell record of cell `along` of a grid line (see cell_source).  Interior
// and mirrored cells take their primitives from Pg when it is given
// (reflection negates the normal momentum and sqrt(rho) u_n and leaves the
// rest unchanged); otherwise they are computed, and stored to Pw when it is
// given and the cell is one of the tile's own (`own`, never a ghost cell).
// Fixed states compute theirs.
template <typename T, int DIM, int DIR>
__device__ __forceinline__ void stage_record(const SweepArgs& a, const T* Ug, const T* Pg, T* Pw, bool own,
                                             long long line_base, int line, int along, int nd, T gamma, T gm1,
                                             T* q)
{
    constexpr int NV = DIM + 2;
    using PL = PrimLayout<DIM>;
    long long g = 0;
    bool flip = false;
    const int fixed = cell_source<DIR>(a, line_base, line, along, nd, g, flip);
    T U[NV], P[PL::NP];
    if (fixed >= 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = pick<T>(a.bc_state[fixed][v], a.bc_state_f[fixed][v]);
        cell_prepare<T, DIM, DIR>(U, gamma, gm1, q);
        return;
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) U[v] = Ug[g + v * a.sv];
    if (Pg != nullptr) {
#pragma unroll
        load_prims<DIM>(Pg, g, P);
    } else {
        cell_prims<T, DIM>(U, gamma, gm1, P);
        if (Pw != nullptr && own) {
            store_prims<DIM>(Pw, g, P);
        }
    }
    if (flip) {
        U[1 + DIR] = -U[1 + DIR];
        P[PL::SU + DIR] = -P[PL::SU + DIR];
    }
    cell_record<T, DIM, DIR>(U, P, q);
}

template <typename T, int DIM>
struct FaceRec {
    // record of a queued WENO face: Roe state, detector, LLF speeds
    static constexpr int NV = DIM + 2;
    static constexpr int U = 0;               // u[DIM]
    static constexpr int C = DIM;
    static constexpr int IC = DIM + 1;
    static constexpr int H = DIM + 2;
    static constexpr int B1 = DIM + 3;
    static constexpr int HQ2 = DIM + 4;
    static constexpr int W = DIM + 5;         // 60 dv^s (Eq. eq28 without the 1/60), NV entries
    static constexpr int AM = W + NV;         // alpha^{u-c} / 2
    static constexpr int A0 = AM + 1;         // alpha^{u} / 2, shear
    static constexpr int AP = AM + 2;         // alpha^{u+c} / 2
    static constexpr int MASK = AM + 3;       // per-field smooth bits (per-field hybrid)
    static constexpr int IRT2 = AM + 4;       // 1 / rho~^2
    static constexpr int NR = AM + 5;
};

// WENO faces are processed in chunks of QC queued faces: 16, or one eighth
// of the tile's faces for tiles of 256 faces and more (in 2D a chunk then
// gives one reconstruction, per face, field and sign, to every thread).
template <int NFACE> struct Chunk { static constexpr int QC = NFACE >= 256 ? NFACE / 8 : 16; };

template <typename T, int DIM, int LINES, int SEG, bool FLAT = false>
struct SweepSmem {
    static constexpr int CELLS = SEG + 6;
    static constexpr int FACES = SEG + 1;
    // a flat tile may hold the end of one line and the start of the next,
    // each with its own three-cell halos: five cells more than one segment
    static constexpr int NCELL = FLAT ? SEG + 11 : LINES * CELLS;
    static constexpr int NFACE = LINES * FACES;
    static constexpr int NQ = CellLayout<DIM>::NQ;
    static constexpr int NV = DIM + 2;
    static constexpr int NR = FaceRec<T, DIM>::NR;
    static constexpr int QC = Chunk<NFACE>::QC;
    static constexpr size_t bytes =
        sizeof(T) * ((size_t)NQ * NCELL + (size_t)NV * NFACE + (size_t)NR * NFACE +
                     (size_t)QC * NV * 2 * 6 + (size_t)QC * NV * 2) +
        sizeof(int) * (size_t)NFACE;
};

// -f_{j-2} + 5 f_{j-1} - 10 f_j + 10 f_{j+1} - 5 f_{j+2} + f_{j+3} as nested
// differences (the negated detector combination of Eq. eq28).  In smooth
// data consecutive differences are close, so each subtraction is exact
// (Sterbenz): the float result carries no cancellation error.
template <typename T>
__device__ __forceinline__ T fifth_difference(T u0, T u1, T u2, T u3, T u4, T u5)
{
    T a0 = u1 - u0, a1 = u2 - u1, a2 = u3 - u2, a3 = u4 - u3, a4 = u5 - u4;
    T b0 = a1 - a0, b1 = a2 - a1, b2 = a3 - a2, b3 = a4 - a3;
    T c0 = b1 - b0, c1 = b2 - b1, c2 = b3 - b2;
    T d0 = c1 - c0, d1 = c2 - c1;
    return d1 - d0;
}

// One tile of the sweep: stage, faces, WENO queue, divergence and output.
// EXACTDET: detector difference by nested differences (mixed precision);
// otherwise the direct six-term combination.  dt is the RK step (COMBINE
// mode only).  Returns true in every thread whose cells failed the
// admissibility check.  Ends with a barrier, so tiles can be chained by one
// CTA (the batched solver) reusing the same shared memory.
//
// Regular tiles hold LINES lines of SEG cells starting at cell seg_blk * SEG.
// A flat tile (LINES = 1, lines of at least SEG cells) holds SEG + 1
// consecutive faces of the sequence of all lines' faces (line after line,
// nd + 1 faces each), starting at face seg_blk * SEG: every tile computes a
// full set of faces, and a tile that reaches the end of a line continues on
// the next one, each piece with its own halo.  line0 and pb are unused then.
template <typename T, int DIM, int DIR, int LINES, int SEG, int NT, bool EXACTDET, bool FLAT = false>
__device__ __forceinline__ bool sweep_tile(const SweepArgs& a, int seg_blk, int line0, int pb, T dt,
                                           unsigned char* smem_raw)
{
    static_assert(!FLAT || LINES == 1, "flat tiles hold one line piece at a time");
    using CL = CellLayout<DIM>;
    using FR = FaceRec<T, DIM>;
    using SM = SweepSmem<T, DIM, LINES, SEG, FLAT>;
    constexpr int NV = DIM + 2;
    constexpr int NQ = CL::NQ;
    constexpr int CELLS = SM::CELLS, FACES = SM::FACES;
    constexpr int NCELL = SM::NCELL, NFACE = SM::NFACE;
    constexpr int NR = FR::NR;
    constexpr int QC = SM::QC;

    T* cq = reinterpret_cast<T*>(smem_raw);     // [NQ][NCELL]  cell records
    T* fh = cq + NQ * NCELL;                    // [NV][NFACE]  face fluxes
    T* fr = fh + NV * NFACE;                    // [NR][NFACE]  WENO face records
    T* fpm = fr + NR * NFACE;                   // [QC][NV][2][6] split fluxes f+-
    T* res = fpm + QC * NV * 2 * 6;             // [QC][NV][2]  reconstructions
    int* queue = reinterpret_cast<int*>(res + QC * NV * 2);
    __shared__ int qcount;
    __shared__ unsigned int wcount;

    const int nd = a.n[DIR];
    const int c0 = seg_blk * SEG;
    const int nline = (DIR == 0) ? a.n[1] : a.n[0];
    const long long sd = DIR == 0 ? 1LL : (DIR == 1 ? a.sy : a.sz);
    const long long sl = DIR == 0 ? a.sy : 1LL;
    const long long sp = DIR == 2 ? a.sy : a.sz;
    const T gamma = pick<T>(a.gamma, a.gamma_f);
    const T gm1 = gamma - T(1);

    const T* Ug = reinterpret_cast<const T*>(a.U);

    // flat tiles: piece A = faces fA0 .. fA0 + nA - 1 of line LA, piece B =
    // faces 0 .. nB - 1 of line LA + 1; in shared memory piece B's cells
    // follow piece A's, so the stencil of face f starts at cell f (piece A)
    // or f + 5 (piece B)
    const int FPL = nd + 1;
    long long LA = 0, Ftot = 0, F0 = 0;
    int fA0 = 0, nA = NFACE, nB = 0;
    if constexpr (FLAT) {
        const long long nl = DIR == 0 ? (long long)a.n[1] * a.n[2]
                                      : (DIR == 1 ? (long long)a.n[0] * a.n[2] : (long long)a.n[0] * a.n[1]);
        Ftot = nl * FPL;
        F0 = (long long)seg_blk * SEG;
        LA = F0 / FPL;
        fA0 = (int)(F0 - LA * FPL);
        nA = FPL - fA0 < NFACE ? FPL - fA0 : NFACE;
        nB = LA + 1 < nl ? NFACE - nA : 0;
    }
    // base address and in-plane index (row j for x sweeps, column i for y/z
    // sweeps) of line li of a flat tile
    auto flat_line = [&](long long li, int& inplane) -> long long {
        if (DIR == 0) {
            const int j = (int)(li % a.n[1]), kk = (int)(li / a.n[1]);
            inplane = j;
            return a.off0 + (long long)j * a.sy + (long long)kk * a.sz;
        } else if (DIR == 1) {
            const int i = (int)(li % a.n[0]), kk = (int)(li / a.n[0]);
            inplane = i;
            return a.off0 + i + (long long)kk * a.sz;
        } else {
            const int i = (int)(li % a.n[0]), j = (int)(li / a.n[0]);
            inplane = i;
            return a.off0 + i + (long long)j * a.sy;
        }
    };

    if (threadIdx.x == 0) { qcount = 0; wcount = 0u; }

    // ---- stage the tile (cells c0-3 .. c0+SEG+2 of LINES lines) --------
    // Cell records from the state and the primitives of the stage (read, or
    // computed and stored for the tile's own cells: those between two of its
    // faces, as the divergence below takes them).
    const T* Pg = reinterpret_cast<const T*>(a.P);
    T* Pw = reinterpret_cast<T*>(a.Pout);
    auto put = [&](int idx, const T (&q)[NQ]) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) cq[k * NCELL + idx] = q[k];
    };
    if constexpr (FLAT) {
        const int nCA = nA + 5, nCB = nB > 0 ? nB + 5 : 0;
        for (int idx = threadIdx.x; idx < nCA + nCB; idx += NT) {
            const bool inA = idx < nCA;
            const int i = (inA ? idx : idx - nCA) - 3;   // cell index relative to the piece's first face
            const bool own = i >= 0 && i <= (inA ? nA : nB) - 2;
            int inplane;
            const long long base = flat_line(inA ? LA : LA + 1, inplane);
            T q[NQ];
            stage_record<T, DIM, DIR>(a, Ug, Pg, Pw, own, base, inplane, inA ? fA0 + i : i, nd, gamma, gm1, q);
            put(idx, q);
        }
    } else if (c0 >= 3 && c0 + SEG + 3 <= nd) {
        // the whole halo is interior (uniform over the block)
        for (int idx = threadIdx.x; idx < NCELL; idx += NT) {
            int l, p;
            if (DIR == 0) { l = idx / CELLS; p = idx - l * CELLS; }
            else { p = idx / LINES; l = idx - p * LINES; }
            const int line = line0 + l;
            if (line < nline) {
                const long long g =
                    a.off0 + (long long)line * sl + (long long)pb * sp + (long long)(c0 - 3 + p) * sd;
                T U[NV], P[PrimLayout<DIM>::NP], q[NQ];
#pragma unroll
                for (int v = 0; v < NV; ++v) U[v] = Ug[g + v * a.sv];
                if (Pg != nullptr) {
                    load_prims<DIM>(Pg, g, P);
                } else {
                    cell_prims<T, DIM>(U, gamma, gm1, P);
                    if (Pw != nullptr && p >= 3 && p < SEG + 3) {
                        store_prims<DIM>(Pw, g, P);
                    }
                }
                cell_record<T, DIM, DIR>(U, P, q);
                put(idx, q);
            }
        }
    } else {
        // a tile at an end of its lines: ghost cells from the boundary conditions
        for (int idx = threadIdx.x; idx < NCELL; idx += NT) {
            int l, p;
            if (DIR == 0) { l = idx / CELLS; p = idx - l * CELLS; }
            else { p = idx / LINES; l = idx - p * LINES; }
            const int line = line0 + l;
            const int along = c0 - 3 + p;
            if (line < nline && along < nd + 3) {
                const bool own = p >= 3 && p < SEG + 3 && along < nd;
                T q[NQ];
                stage_record<T, DIM, DIR>(a, Ug, Pg, Pw, own, a.off0 + (long long)line * sl + (long long)pb * sp,
                                          line, along, nd, gamma, gm1, q);
                put(idx, q);
            }
        }
    }
    __syncthreads();

    // shared-memory order follows the global order: along-the-line for x
    // sweeps, across the lines (x fastest) for y/z sweeps; consecutive
    // threads read consecutive words in both cases
    auto cidx = [](int l, int p) -> int { return DIR == 0 ? l * CELLS + p : p * LINES + l; };
    auto fdec = [&](int f, int& l, int& p) {
        if constexpr (FLAT) { l = 0; p = f < nA ? f : f + 5; }
        else if (DIR == 0) { l = f / FACES; p = f - l * FACES; }
        else { p = f / LINES; l = f - p * LINES; }
    };

    // sigma^s < eps_h  <=>  |60 dv^s| < 60 sqrt(eps_h) rho~ (both sides >= 0)
    const T slim = pick<T>(a.slim, a.slim_f);
    const T lam_scale = pick<T>(a.c_lambda * (1.0 / 3600.0), a.lam_scale_f);
    const int lane = threadIdx.x & 31;
    unsigned int my_weno = 0;

    // ---- phase 1: detector, linear upwind faces, queue of WENO faces -----
    for (int f0 = 0; f0 < NFACE; f0 += NT) {
        const int f = f0 + threadIdx.x;
        int l = 0, p = 0;
        bool valid = f < NFACE;
        if (valid) {
            fdec(f, l, p);
            if constexpr (FLAT) valid = f < nA + nB;
            else valid = (line0 + l < nline) && (c0 + p <= nd);
        }
        bool weno = false;
        if (valid) {
            auto ga = [&](int k) -> T { return cq[k * NCELL + cidx(l, p + 2)]; };
            auto gb = [&](int k) -> T { return cq[k * NCELL + cidx(l, p + 3)]; };
            const Roe<T, DIM> r = roe_state<T, DIM>(ga, gb, gm1);
            // Eq. eq28 without the 1/60: w = L (U_{j-2} - 5U_{j-1} + 10U_j - 10U_{j+1} + 5U_{j+2} - U_{j+3})
            T dU[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const int k = CL::U + v;
                const T u0 = cq[k * NCELL + cidx(l, p + 0)];
                const T u1 = cq[k * NCELL + cidx(l, p + 1)];
                const T u2 = cq[k * NCELL + cidx(l, p + 2)];
                const T u3 = cq[k * NCELL + cidx(l, p + 3)];
                const T u4 = cq[k * NCELL + cidx(l, p + 4)];
                const T u5 = cq[k * NCELL + cidx(l, p + 5)];
                if (EXACTDET) dU[v] = -fifth_difference(u0, u1, u2, u3, u4, u5);
                else dU[v] = fmaT(T(10), u2 - u3, fmaT(T(5), u4 - u1, u0 - u5));
            }
            T w[NV];
            proj_all<T, DIM, DIR>(r, dU, w);
            const T lim = slim * r.rt;
            int fmask = 0;
#pragma unroll
            for (int s = 0; s < NV; ++s) fmask |= abs_lt(w[s], lim) ? (1 << s) : 0;
            const bool smooth = a.hybrid != 0 && fmask == (1 << NV) - 1;
            // splitting speeds: LLF max over the six stencil cells, global
            // LF maxima, or the Roe-average eigenvalues
            T am, a0, ap;
            if (a.split == SPLIT_LLF) {
                am = cq[CL::LM * NCELL + cidx(l, p)];
                a0 = cq[CL::L0 * NCELL + cidx(l, p)];
                ap = cq[CL::LP * NCELL + cidx(l, p)];
#pragma unroll
                for (int m = 1; m < 6; ++m) {
                    am = max_nn(am, cq[CL::LM * NCELL + cidx(l, p + m)]);
                    a0 = max_nn(a0, cq[CL::L0 * NCELL + cidx(l, p + m)]);
                    ap = max_nn(ap, cq[CL::LP * NCELL + cidx(l, p + m)]);
                }
            } else if (a.split == SPLIT_RF) {
                am = absT(r.u[DIR] - r.c);
                a0 = absT(r.u[DIR]);
                ap = absT(r.u[DIR] + r.c);
            } else {
                am = T(__longlong_as_double((long long)a.alpha_g[0]));
                a0 = T(__longlong_as_double((long long)a.alpha_g[1]));
                ap = T(__longlong_as_double((long long)a.alpha_g[2]));
            }
            if (smooth) {
                // Eq. linearupwind: [central six-point flux + sum_s R^s alpha^s (60 dv^s)] / 60
                T Fo[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const int k = CL::F + v;
                    const T f05 = cq[k * NCELL + cidx(l, p + 0)] + cq[k * NCELL + cidx(l, p + 5)];
                    const T f14 = cq[k * NCELL + cidx(l, p + 1)] + cq[k * NCELL + cidx(l, p + 4)];
                    const T f23 = cq[k * NCELL + cidx(l, p + 2)] + cq[k * NCELL + cidx(l, p + 3)];
                    Fo[v] = fmaT(T(37), f23, fmaT(T(-8), f14, f05));
                }
                ups_dissipation_add<T, DIM, DIR>(r, dU, w, am, a0, ap, Fo);
                // face fluxes are kept times 60; the divergence scales by dx/60
#pragma unroll
                for (int v = 0; v < NV; ++v) fh[v * NFACE + f] = Fo[v];
            } else {
                weno = true;
#pragma unroll
                for (int k = 0; k < DIM; ++k) fr[(FR::U + k) * NFACE + f] = r.u[k];
                fr[FR::C * NFACE + f] = r.c;
                fr[FR::IC * NFACE + f] = r.ic;
                fr[FR::H * NFACE + f] = r.H;
                fr[FR::B1 * NFACE + f] = r.b1;
                fr[FR::HQ2 * NFACE + f] = r.hq2;
                // the regularization parameters of Eq. eq27, eq29 are formed
                // in phase 2 from w and 1 / rho~^2 (few lanes of this warp
                // take this branch)
#pragma unroll
                for (int s = 0; s < NV; ++s) fr[(FR::W + s) * NFACE + f] = w[s];
                fr[FR::IRT2 * NFACE + f] = Ar<T>::rcp_f(r.rt * r.rt);
                // half splitting speeds (Eq. flxuspliting: f+- = (g +- alpha v) / 2)
                fr[FR::AM * NFACE + f] = halve(am);
                fr[FR::A0 * NFACE + f] = halve(a0);
                fr[FR::AP * NFACE + f] = halve(ap);
                fr[FR::MASK * NFACE + f] = T(a.hybrid == 2 ? fmask : 0);
            }
            // a face is owned by the tile left of it, the last face by the last tile
            int face = c0 + p;
            bool owned = (p < SEG) || (face == nd);
            if constexpr (FLAT) {
                face = f < nA ? fA0 + f : f - nA;
                owned = (f < SEG) || (F0 + f == Ftot - 1);
            }
            if (owned) {
                if (weno) ++my_weno;
                if (a.flags != nullptr) {
                    int line = line0 + l, pbf = pb;
                    if constexpr (FLAT) {
                        const long long li = f < nA ? LA : LA + 1;
                        if (DIR == 0) { line = (int)(li % a.n[1]); pbf = (int)(li / a.n[1]); }
                        else { line = (int)(li % a.n[0]); pbf = (int)(li / a.n[0]); }
                    }
                    long long fidx;
                    if (DIR == 0) fidx = ((long long)pbf * a.n[1] + line) * (long long)(nd + 1) + face;
                    else if (DIR == 1) fidx = ((long long)pbf * (nd + 1) + face) * (long long)a.n[0] + line;
                    else fidx = ((long long)face * a.n[1] + pbf) * (long long)a.n[0] + line;
                    a.flags[fidx] = weno ? 0 : 1;
                }
            }
        }
        const unsigned int mask = __ballot_sync(0xffffffffu, weno);
        if (mask) {
            int base = 0;
            const int leader = __ffs(mask) - 1;
            if (lane == leader) base = atomicAdd(&qcount, __popc(mask));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (weno) queue[base + __popc(mask & ((1u << lane) - 1u))] = f;
        }
    }
    if (my_weno) atomicAdd(&wcount, my_weno);
    __syncthreads();

    // ---- phase 2: characteristic regularized WENO-IS flux of queued faces --
    const int nq = qcount;
    const T eps = pick<T>(a.eps, a.eps_f);
    for (int q0 = 0; q0 < nq; q0 += QC) {
        const int qc = nq - q0 < QC ? nq - q0 : QC;
        // 2a: project U_m and F_m of the six stencil cells (Eq. eqchara) and
        //     split them (Eq. flxuspliting); one work item per (face, cell)
        for (int it = threadIdx.x; it < qc * 6; it += NT) {
            const int q = it / 6, m = it - (it / 6) * 6;
            const int f = queue[q0 + q];
            int l, p;
            fdec(f, l, p);
            Roe<T, DIM> r;
#pragma unroll
            for (int k = 0; k < DIM; ++k) r.u[k] = fr[(FR::U + k) * NFACE + f];
            r.ic = fr[FR::IC * NFACE + f];
            r.b1 = fr[FR::B1 * NFACE + f];
            r.hq2 = fr[FR::HQ2 * NFACE + f];
            const T am = fr[FR::AM * NFACE + f];
            const T a0 = fr[FR::A0 * NFACE + f];
            const T ap = fr[FR::AP * NFACE + f];
            const int ci = cidx(l, p + m);
            T xu[NV], xf[NV], wv[NV], wg[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                xu[v] = cq[(CL::U + v) * NCELL + ci];
                xf[v] = cq[(CL::F + v) * NCELL + ci];
            }
            proj_all<T, DIM, DIR>(r, xu, wv);
            proj_all<T, DIM, DIR>(r, xf, wg);
#pragma unroll
            for (int s = 0; s < NV; ++s) {
                const T al = s == 0 ? am : (s == NV - 1 ? ap : a0);
                const T h = halve(wg[s]);
                const T k = al * wv[s];   // al holds alpha / 2
                // f+ in stencil order j-2 .. j+3, f- mirrored (j+3 .. j-2), so
                // that both signs take the same call in 2b (neighbouring lanes
                // hold the two signs and would otherwise diverge)
                fpm[((q * NV + s) * 2 + 0) * 6 + m] = h + k;
                fpm[((q * NV + s) * 2 + 1) * 6 + (5 - m)] = h - k;
            }
        }
        __syncthreads();
        // 2b: one reconstruction per (face, field, sign): Eq. eq6, eq11, eq18,
        //     eq8-r; the minus part on the mirrored stencil j+3 .. j-1 (stored
        //     mirrored by 2a)
        for (int it = threadIdx.x; it < qc * NV * 2; it += NT) {
            const int q = it / (2 * NV);
            const int rem = it - q * (2 * NV);
            const int s = rem >> 1, sg = rem & 1;
            const int f = queue[q0 + q];
            // Eq. eq27, eq29: lambda^s = c (dv^s / rho~)^2 = c w_s^2 / (3600 rho~^2)
            const T ws = fr[(FR::W + s) * NFACE + f];
            const T lam = lam_scale * (ws * ws) * fr[FR::IRT2 * NFACE + f];
            // per-field hybrid: the linear scheme for a smooth field
            const int fm_bits = (int)fr[FR::MASK * NFACE + f];
            const int wm = (fm_bits >> s) & 1 ? W_LINEAR : a.wmode;
            const T* v = fpm + ((q * NV + s) * 2 + sg) * 6;
            res[(q * NV + s) * 2 + sg] = recon<T>(v[0], v[1], v[2], v[3], v[4], lam, eps, wm);
        }
        __syncthreads();
        // 2c: Eq. reconstruction1 and the back-projection Eq. reconstruction2,
        //     one work item per (face, conserved variable)
        for (int it = threadIdx.x; it < qc * NV; it += NT) {
            const int q = it / NV, v = it - (it / NV) * NV;
            const int f = queue[q0 + q];
            Roe<T, DIM> r;
#pragma unroll
            for (int k = 0; k < DIM; ++k) r.u[k] = fr[(FR::U + k) * NFACE + f];
            r.c = fr[FR::C * NFACE + f];
            r.H = fr[FR::H * NFACE + f];
            r.hq2 = fr[FR::HQ2 * NFACE + f];
            T wch[NV];
#pragma unroll
            for (int s = 0; s < NV; ++s) wch[s] = res[(q * NV + s) * 2] + res[(q * NV + s) * 2 + 1];
            fh[v * NFACE + f] = T(60) * back_proj_row<T, DIM, DIR>(r, wch, v);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && a.weno_count != nullptr && wcount != 0u)
        atomicAdd(a.weno_count, (unsigned long long)wcount);

    // ---- flux divergence and output ---------------------------------------
    const T inv_dx = pick<T>(a.inv_dx * (1.0 / 60.0), a.inv_dx_f);
    T* outp = reinterpret_cast<T*>(a.out);
    T* accp = reinterpret_cast<T*>(a.acc);
    const T* Unp = reinterpret_cast<const T*>(a.Un);
    const T rka = pick<T>(a.rk_a, a.rk_a_f), rkb = pick<T>(a.rk_b, a.rk_b_f);
    const T acs = pick<T>(a.acc_scale, a.acc_scale_f);
    bool bad = false;
    for (int idx = threadIdx.x; idx < LINES * SEG; idx += NT) {
        int l, p;
        if (DIR == 0) { l = idx / SEG; p = idx - l * SEG; }
        else { p = idx / LINES; l = idx - p * LINES; }
        long long g;
        int fl, fr_, cpos;   // left and right face, stencil start of the left face
        if constexpr (FLAT) {
            // the cell between faces idx and idx + 1 of the same piece
            const bool inA = idx + 1 < nA;
            if (!inA && (idx < nA || idx + 1 >= nA + nB)) continue;   // line junction or past the end
            int inplane;
            g = flat_line(inA ? LA : LA + 1, inplane) + (long long)(inA ? fA0 + idx : idx - nA) * sd;
            fl = idx;
            fr_ = idx + 1;
            cpos = inA ? idx : idx + 5;
        } else {
            const int line = line0 + l;
            const int cell = c0 + p;
            if (line >= nline || cell >= nd) continue;
            g = a.off0 + (long long)line * sl + (long long)pb * sp + (long long)cell * sd;
            fl = DIR == 0 ? l * FACES + p : p * LINES + l;
            fr_ = DIR == 0 ? fl + 1 : fl + LINES;
            cpos = p;
        }
        if (a.mode == MODE_ACC_SET) {
            // the flux difference unscaled: the sweep that reads the
            // accumulator multiplies it by acc_scale
#pragma unroll
            for (int v = 0; v < NV; ++v) accp[g + v * a.sv] = fh[v * NFACE + fl] - fh[v * NFACE + fr_];
            continue;
        }
        T rv[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) rv[v] = (fh[v * NFACE + fl] - fh[v * NFACE + fr_]) * inv_dx;
        if (a.mode == MODE_ACC_ADD) {
#pragma unroll
            for (int v = 0; v < NV; ++v) accp[g + v * a.sv] = fmaT(accp[g + v * a.sv], acs, rv[v]);
        } else if (a.mode == MODE_RHS) {
#pragma unroll
            for (int v = 0; v < NV; ++v) outp[g + v * a.sv] = accp ? fmaT(accp[g + v * a.sv], acs, rv[v]) : rv[v];
        } else {
            const int ci = FLAT ? cpos + 3 : cidx(l, cpos + 3);
            T nu[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                T tot = rv[v];
                if (accp) tot = fmaT(accp[g + v * a.sv], acs, tot);
                T val = rkb * fmaT(dt, tot, cq[(CL::U + v) * NCELL + ci]);
                if (rka != T(0)) val = fmaT(rka, Unp[g + v * a.sv], val);
                nu[v] = val;
                outp[g + v * a.sv] = val;
            }
            // admissibility: rho > 0, p > 0  <=>  2 rho E > |m|^2, finite
            T m2 = T(0);
#pragma unroll
            for (int k = 0; k < DIM; ++k) m2 = fmaT(nu[1 + k], nu[1 + k], m2);
            const T chk = T(2) * nu[0] * nu[DIM + 1] - m2;
            if (!(nu[0] > T(0)) || !(chk > T(0)) || !isfinite(chk)) bad = true;
        }
    }
    __syncthreads();
    return bad;
}

template <typename T, int DIM, int DIR, int LINES, int SEG, int NT, bool EXACTDET, bool FLAT = false>
__global__ void __launch_bounds__(NT, NT <= 128 ? 4 : 2) k_sweep(SweepArgs a)
{
    pdl_enter();
    if (a.tm != nullptr) {
        if (a.tm->status != 0 || !(a.tm->dt > 0.0)) return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int seg_blk, line0, pb;
    if (FLAT) { seg_blk = blockIdx.x; line0 = 0; pb = 0; }
    else if (DIR == 0) { seg_blk = blockIdx.x; line0 = blockIdx.y * LINES; pb = blockIdx.z; }
    else if (DIR == 1) { seg_blk = blockIdx.y; line0 = blockIdx.x * LINES; pb = blockIdx.z; }
    else { seg_blk = blockIdx.z; line0 = blockIdx.x * LINES; pb = blockIdx.y; }
    const T dt = a.mode == MODE_COMBINE ? T(a.tm->dt) : T(0);
    const bool bad = sweep_tile<T, DIM, DIR, LINES, SEG, NT, EXACTDET, FLAT>(a, seg_blk, line0, pb, dt, smem_raw);
    if (bad) atomicOr(&a.tm->status, 1);
}

// ---------------------------------------------------------------- ghosts
// Boundary conditions of one direction, as the adjoint's ghost-gradient
// mapping (k_ghost_adj) reads them.
struct GhostArgs {
    void* U;
    int dir;
    int n[3];
    long long sy, sz, sv, off0;
    int bc_lo, bc_hi;
    double bc_state[2][5];
    double lo0, dx0;     // x-axis geometry for the DMR boundaries
    double lo1, dx1;     // y-axis geometry for the jet inflow
    DevTime* tm;         // stage time from tm (t + stage_c dt), or t_fixed
    double stage_c, t_fixed;
};

// ------------------------------------------------------- CFL reduction
struct CflArgs {
    const void* U;
    int n[3];
    long long sy, sz, sv, off0;
    double inv_dx[3];
    double gamma;
    DevTime* tm;
    int parts;    // k_cfl: x-parts per grid row (rows x parts blocks of work)
};

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = maxT(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// CFL wave-speed sum sum_d (|u_d| + c) / dx_d of one cell; false if the cell
// is not admissible (rho <= 0, p <= 0 or non-finite).  Shared by the grid
// reduction and the batched solver so both take identical time steps.
template <typename T, int DIM>
__device__ __forceinline__ bool cell_speed(const T* u, T gamma, const T* inv_dx, T& s)
{
    const T gm1 = gamma - T(1);
    const T irho = Ar<T>::rcp_f(u[0]);
    T ke2 = T(0);
    T vel[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) { vel[d] = u[1 + d] * irho; ke2 = fmaT(u[1 + d], vel[d], ke2); }
    const T p = gm1 * fmaT(T(-0.5), ke2, u[DIM + 1]);
    const T c2 = gamma * p * irho;
    const T c = c2 * Ar<T>::rsqrt_(c2);   // NaN for p <= 0, rejected below
    s = T(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) s = fmaT(absT(vel[d]) + c, inv_dx[d], s);
    return (u[0] > T(0)) && (p > T(0)) && isfinite(s);
}

// dt = CFL / smax clipped to t_end (the clipped step lands exactly on t_end)
__device__ __forceinline__ double cfl_step(double cfl, double smax, double t, double t_end, int* clipped)
{
    double dt = 0.0;
    *clipped = 0;
    if (t < t_end) {
        if (smax > 0.0) dt = cfl / smax;
        if (t + dt >= t_end) { dt = t_end - t; *clipped = 1; }
        if (!(dt > 0.0)) { dt = 0.0; *clipped = 0; }
    }
    return dt;
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_cfl(CflArgs a)
{
    pdl_enter();
    constexpr int NV = DIM + 2;
    if (a.tm->status != 0) return;
    const T* U = reinterpret_cast<const T*>(a.U);
    const int nx = a.n[0], ny = a.n[1];
    const long long rows = (long long)ny * a.n[2];
    const T gamma = T(a.gamma);
    T idx_[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) idx_[k] = T(a.inv_dx[k]);
    // work unit: one of `parts` x-ranges of one grid row (row indices are
    // decomposed once per unit, not per cell); the running max of the
    // non-negative speeds is exact in the storage precision
    const int span = (nx + a.parts - 1) / a.parts;
    T smax_t = T(0);
    bool bad = false;
    for (long long c = blockIdx.x; c < rows * a.parts; c += gridDim.x) {
        const long long row = c / a.parts;
        const int part = (int)(c - row * a.parts);
        const int j = (int)(row % ny), k = (int)(row / ny);
        const long long gr = a.off0 + (long long)j * a.sy + (long long)k * a.sz;
        const int x1 = min(nx, (part + 1) * span);
        for (int i = part * span + threadIdx.x; i < x1; i += blockDim.x) {
            T u[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) u[v] = U[gr + i + v * a.sv];
            T s;
            if (!cell_speed<T, DIM>(u, gamma, idx_, s)) bad = true;
            else smax_t = max_nn(smax_t, s);
        }
    }
    double smax = (double)smax_t;
    __shared__ double red[8];
    smax = warp_max(smax);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = smax;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_max(v);
        if (threadIdx.x == 0 && v > 0.0)
            atomicMax(&a.tm->smax_bits, (unsigned long long)__double_as_longlong(v));
    }
    if (bad) atomicOr(&a.tm->status, 1);
}

// global Lax-Friedrichs speeds (Sec. 2.4 step (4), l = the whole domain):
// per direction d, max over interior cells of |u_d - c|, |u_d|, |u_d + c|,
// as bits of non-negative doubles (out[3 d + k], zeroed beforehand)
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_lf_alpha(CflArgs a, unsigned long long* out)
{
    pdl_enter();
    constexpr int NV = DIM + 2;
    if (a.tm != nullptr && (a.tm->status != 0 || !(a.tm->dt > 0.0))) return;
    const T* U = reinterpret_cast<const T*>(a.U);
    const long long nx = a.n[0], ny = a.n[1];
    const long long total = nx * ny * (long long)a.n[2];
    const T gamma = T(a.gamma), gm1 = gamma - T(1);
    double mx[3 * DIM];
#pragma unroll
    for (int q = 0; q < 3 * DIM; ++q) mx[q] = 0.0;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
        const long long i = id % nx, j = (id / nx) % ny, k = id / (nx * ny);
        const long long g = a.off0 + i + j * a.sy + k * a.sz;
        T u[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = U[g + v * a.sv];
        T q[CellLayout<DIM>::NQ];
        const T irho = Ar<T>::rcp(u[0]);
        T ke2 = T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) ke2 = fmaT(u[1 + d], u[1 + d] * irho, ke2);
        const T p = gm1 * fmaT(T(-0.5), ke2, u[DIM + 1]);
        const T c = Ar<T>::sqrt_(gamma * p * irho);
        (void)q;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const T un = u[1 + d] * irho;
            mx[3 * d + 0] = maxT(mx[3 * d + 0], (double)absT(un - c));
            mx[3 * d + 1] = maxT(mx[3 * d + 1], (double)absT(un));
            mx[3 * d + 2] = maxT(mx[3 * d + 2], (double)absT(un + c));
        }
    }
#pragma unroll
    for (int q = 0; q < 3 * DIM; ++q) {
        const double v = warp_max(mx[q]);
        if ((threadIdx.x & 31) == 0 && v > 0.0) atomicMax(&out[q], (unsigned long long)__double_as_longlong(v));
    }
}

// dt = CFL / smax clipped to t_end; resets the reduction cell
// smax_floor: wave-speed sum of the fixed boundary states (they enter the
// domain through the ghost cells)
static __global__ void k_dt(DevTime* tm, double cfl, double smax_floor)
{
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double dt = 0.0;
    int clipped = 0;
    if (tm->status == 0) {
        const double smax = maxT(__longlong_as_double((long long)tm->smax_bits), smax_floor);
        dt = cfl_step(cfl, smax, tm->t, tm->t_end, &clipped);
    }
    tm->dt = dt;
    tm->clipped = clipped;
    tm->smax_bits = 0ull;
    // boundary times of the three stages (Shu-Osher RK3: t, t + dt, t + dt/2)
    tm->xs_top[0] = dmr_shock_x(tm->t);
    tm->xs_top[1] = dmr_shock_x(tm->t + dt);
    tm->xs_top[2] = dmr_shock_x(tm->t + 0.5 * dt);
}

// target time for the steps that follow on the stream
static __global__ void k_set_tend(DevTime* tm, double t_end)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) tm->t_end = t_end;
}

static __global__ void k_post(DevTime* tm)
{
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (tm->status == 0 && tm->dt > 0.0) {
        tm->t = tm->clipped ? tm->t_end : tm->t + tm->dt;
        tm->steps += 1;
    }
    tm->dt = 0.0;
}

// ------------------------------------------------------- conserved totals
struct TotArgs {
    const void* U;
    int n[3];
    long long sy, sz, sv, off0;
    double* partial;   // [gridDim.x][NV]
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_totals(TotArgs a)
{
    constexpr int NV = DIM + 2;
    const T* U = reinterpret_cast<const T*>(a.U);
    const long long nx = a.n[0], ny = a.n[1];
    const long long total = nx * ny * (long long)a.n[2];
    double s[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) s[v] = 0.0;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
        const long long i = id % nx, j = (id / nx) % ny, k = id / (nx * ny);
        const long long g = a.off0 + i + j * a.sy + k * a.sz;
#pragma unroll
        for (int v = 0; v < NV; ++v) s[v] += (double)U[g + v * a.sv];
    }
    __shared__ double red[8][NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const double w = warp_sum(s[v]);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][v] = w;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double w = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) w += red[q][threadIdx.x];
        a.partial[blockIdx.x * NV + threadIdx.x] = w;
    }
}

// sum of the per-block partials in a fixed order, times the cell volume
static __global__ void k_totals_final(const double* partial, int nblk, int nv, double dV, double* out)
{
    const int v = threadIdx.x;
    if (v >= nv) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[b * nv + v];
    out[v] = s * dV;
}

// --------------------------------------- interior <-> ghosted layout copies
// One work unit is up to blockDim.x consecutive cells of one row (variable
// v, rows j, k) of the interior-only array, whose index is row * nx + i with
// row = (v nz + k) ny + j.  The index arithmetic is done once per unit; the
// threads of a block copy consecutive cells, coalesced on both sides.
template <typename T>
__global__ void k_pack(const T* src, T* dst, int nv, int nx, int ny, int nz, long long sy, long long sz,
                       long long sv, long long off0, int to_ghosted)
{
    const int chunks = (nx + blockDim.x - 1) / blockDim.x;
    const long long plane = (long long)ny * nz;
    const long long units = (long long)nv * plane * chunks;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const long long row = u / chunks;
        const int i = (int)(u - row * chunks) * blockDim.x + threadIdx.x;
        if (i >= nx) continue;
        const long long v = row / plane, jk = row - v * plane;
        const long long k = jk / ny, j = jk - k * ny;
        const long long lin = row * nx + i;
        const long long g = off0 + i + j * sy + k * sz + v * sv;
        if (to_ghosted) dst[g] = src[lin];
        else dst[lin] = src[g];
    }
}

}  // namespace wis
