// Hand-written adjoint (vector-Jacobian product) of the semi-discrete
// operator dU/dt = -sum_d (F_{j+1/2} - F_{j-1/2}) / dx_d.
//
// For a cotangent w (one value per cell and variable) the face flux F_f of
// direction d receives the cotangent phi_f = (w_{j+1} - w_j) / dx_d (w = 0
// outside the domain), and gU = sum_f (dF_f / dU_stencil)^T phi_f.  Every
// face recomputes its forward quantities (Roe state, detector, LLF speeds,
// projections, reconstructions: nothing is stored by the forward pass) and
// then runs the reverse of each step:
//   back-projection (Eq. reconstruction2)  -> back_proj_adj
//   reconstruction (Eq. eq6, eq11, eq18, eq8-r) -> recon_adj
//   splitting and projection (Eq. flxuspliting, eqchara) -> proj_all_adj
//   regularization parameter (Eq. eq27-29) and detector (Eq. eq28)
//   Roe average (Sec. 2.4 step (1)) -> roe_adj
//   cell primitives and physical flux -> cell_adj
// The hybrid flag and the cell that attains each LLF maximum are held at
// their forward values (first index on ties): the operator is piecewise
// smooth and this is the derivative of the active piece.
//
// Accumulation is deterministic: a tile of SEG cells recomputes the SEG + 5
// faces that touch its cells, writes each face's contribution to its six
// stencil cells in shared memory, and gathers them per cell in face order.
// A linear-upwind face stores two bar vectors, of the central-flux sum and
// of the detector difference, and the gather applies their fixed stencil
// weights; a WENO face stores U and F bars for each of its six cells.  Every
// face adds Roe-field bars for its two neighbours and one bar per LLF speed
// for the cell attaining it.
//
// Each direction runs in two passes over the same tiles.  Pass 0 takes the
// linear-upwind faces, writes (or adds) the gradient, and flags each tile
// that has a WENO face among the faces it recomputes.  Pass 1 runs on the
// flagged tiles only, takes their WENO faces and adds their contributions.
// The WENO reverse needs the registers of the 6 x nvar projections and
// their bars; keeping it out of pass 0 lets the common linear-upwind tiles
// run with far fewer registers and more resident warps.
// Contributions to ghost cells go to a per-line buffer that a second kernel
// maps back through the boundary conditions.
#pragma once

#include "weno_kernels.cuh"

namespace wis {

// q sgn(x): q with x's sign applied, zero where x is zero; for double on the
// integer pipes (the FP64 pipe bounds the adjoint), the same value as the
// product for finite q (a zero result may differ in its sign only)
__device__ __forceinline__ double times_sign(double q, double x)
{
    const long long xb = __double_as_longlong(x);
    const long long r = __double_as_longlong(q) ^ (xb & (long long)0x8000000000000000ULL);
    return (xb & 0x7fffffffffffffffLL) == 0 ? 0.0 : __longlong_as_double(r);
}
__device__ __forceinline__ float times_sign(float q, float x)
{
    return x > 0.0f ? q : (x < 0.0f ? -q : 0.0f);
}

// record bars of one cell (NQ entries, same layout as CellLayout) -> dU;
// isq = 1/sqrt(rho), ic = 1/c, the pressure p and the sound speed c as
// cell_prims computed them for the forward record
template <typename T, int DIM, int DIR>
__device__ __forceinline__ void cell_adj(const T* U, T gamma, T isq, T ic, T p, T c, const T* qb, T* Ub)
{
    using CL = CellLayout<DIM>;
    constexpr int NV = DIM + 2;
    const T gm1 = gamma - T(1);
    const T rho = U[0];
    const T irho = isq * isq;
    T m2 = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) m2 = fmaT(U[1 + k], U[1 + k], m2);
    const T E = U[DIM + 1];
    const T un = U[1 + DIR] * irho;
    const T Ep = E + p;

#pragma unroll
    for (int v = 0; v < NV; ++v) Ub[v] = qb[CL::U + v];
    T unb = T(0), cb = T(0), isqb = T(0), Epb = T(0), pb = T(0), irhob = T(0), m2b = T(0);
    // |un - c|, |un|, |un + c|: the bars take the signs of their arguments
    const T lm = times_sign(qb[CL::LM], un - c), lp = times_sign(qb[CL::LP], un + c);
    unb += lm; cb -= lm;
    unb += times_sign(qb[CL::L0], un);
    unb += lp; cb += lp;
    Ub[0] += qb[CL::SQ] * isq; isqb += qb[CL::SQ] * rho;
    Epb += qb[CL::SH] * isq; isqb += qb[CL::SH] * Ep;
#pragma unroll
    for (int k = 0; k < DIM; ++k) { Ub[1 + k] += qb[CL::SU + k] * isq; isqb += qb[CL::SU + k] * U[1 + k]; }
    Epb += qb[CL::F + DIM + 1] * un; unb += qb[CL::F + DIM + 1] * Ep;
#pragma unroll
    for (int k = 0; k < DIM; ++k) { Ub[1 + k] += qb[CL::F + 1 + k] * un; unb += qb[CL::F + 1 + k] * U[1 + k]; }
    pb += qb[CL::F + 1 + DIR];
    Ub[1 + DIR] += qb[CL::F + 0];
    Ub[DIM + 1] += Epb; pb += Epb;
    Ub[1 + DIR] += unb * irho; irhob += unb * U[1 + DIR];
    // c = sqrt(gamma p irho): dc = gamma (irho dp + p dirho) / (2 c)
    const T cg = halve(cb) * ic * gamma;
    pb = fmaT(cg, irho, pb); irhob = fmaT(cg, p, irhob);
    // p = gm1 (E - irho m2 / 2)
    const T pg = pb * gm1, hpg = halve(pg);
    Ub[DIM + 1] += pg; irhob = fmaT(-hpg, m2, irhob); m2b = -hpg * irho;
    // m2 = |m|^2, irho = isq^2, isq = rho^-1/2
    const T m2b2 = m2b + m2b;
#pragma unroll
    for (int k = 0; k < DIM; ++k) Ub[1 + k] = fmaT(U[1 + k], m2b2, Ub[1 + k]);
    isqb = fmaT(isq + isq, irhob, isqb);
    Ub[0] = fmaT(isqb, -halve(isq) * irho, Ub[0]);
}

template <typename T, int DIM> struct RoeBar {
    T u[DIM];
    T c, ic, H, b1, hq2, rt;
};

template <typename T, int DIM>
__device__ __forceinline__ void zero(RoeBar<T, DIM>& b)
{
#pragma unroll
    for (int k = 0; k < DIM; ++k) b.u[k] = T(0);
    b.c = b.ic = b.H = b.b1 = b.hq2 = b.rt = T(0);
}

// adjoint of w = L x (proj_all): accumulates xb and rb
template <typename T, int DIM, int DIR>
__device__ __forceinline__ void proj_all_adj(const Roe<T, DIM>& r, const T* x, const T* wb, T* xb,
                                             RoeBar<T, DIM>& rb)
{
    constexpr int LAST = DIM + 1;
    T dot = r.u[0] * x[1];
#pragma unroll
    for (int k = 1; k < DIM; ++k) dot = fmaT(r.u[k], x[1 + k], dot);
    const T y = fmaT(r.hq2, x[0], x[DIM + 1]) - dot;
    const T z = fmaT(r.u[DIR], x[0], -x[1 + DIR]);
    const T t1b = halve(wb[0] + wb[LAST]) - wb[1];
    const T ab = halve(wb[0] - wb[LAST]);
    int s = 2;
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
        if (t == DIR) continue;
        xb[1 + t] += wb[s];
        xb[0] -= wb[s] * r.u[t];
        rb.u[t] -= wb[s] * x[0];
        ++s;
    }
    xb[0] += wb[1];
    const T zb = ab * r.ic;
    rb.ic += ab * z;
    rb.u[DIR] += zb * x[0];
    xb[0] += zb * r.u[DIR];
    xb[1 + DIR] -= zb;
    rb.b1 += t1b * y;
    const T yb = t1b * r.b1;
    rb.hq2 += yb * x[0];
    xb[0] += yb * r.hq2;
    xb[DIM + 1] += yb;
#pragma unroll
    for (int k = 0; k < DIM; ++k) { rb.u[k] -= yb * x[1 + k]; xb[1 + k] -= yb * r.u[k]; }
}

// adjoint of out = R w (back_proj_add): sets wb, accumulates rb
template <typename T, int DIM, int DIR>
__device__ __forceinline__ void back_proj_adj(const Roe<T, DIM>& r, const T* w, const T* ob, T* wb,
                                              RoeBar<T, DIM>& rb)
{
    constexpr int LAST = DIM + 1;
    const T sum = w[0] + w[1] + w[LAST];
    const T dif = w[LAST] - w[0];
    const T oE = ob[LAST];
    T sumb = ob[0];
#pragma unroll
    for (int k = 0; k < DIM; ++k) { sumb = fmaT(ob[1 + k], r.u[k], sumb); rb.u[k] += ob[1 + k] * sum; }
    const T difb = (ob[1 + DIR] + oE * r.u[DIR]) * r.c;
    rb.c += (ob[1 + DIR] + oE * r.u[DIR]) * dif;
    rb.u[DIR] += oE * r.c * dif;
#pragma unroll
    for (int s = 0; s <= LAST; ++s) wb[s] = T(0);
    int s = 2;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        if (k == DIR) continue;
        wb[s] = ob[1 + k] + oE * r.u[k];
        rb.u[k] += oE * w[s];
        ++s;
    }
    rb.H += oE * (w[0] + w[LAST]);
    rb.hq2 += oE * w[1];
    wb[0] += oE * r.H + sumb - difb;
    wb[1] += oE * r.hq2 + sumb;
    wb[LAST] += oE * r.H + sumb + difb;
}

// adjoint of the Roe average; gab/gbb: bars of the Roe fields of cells j and
// j+1, relative to CL::SU (sqrt(rho) u at 0 .. DIM-1, sqrt(rho) H at DIM,
// sqrt(rho) at DIM + 1)
template <typename T, int DIM, typename GA, typename GB>
__device__ __forceinline__ void roe_adj(GA get_a, GB get_b, T gamma, const Roe<T, DIM>& r, RoeBar<T, DIM> rb,
                                        T* gab, T* gbb)
{
    using CL = CellLayout<DIM>;
    const T gm1 = gamma - T(1);
    const T sa = get_a(CL::SQ), sb = get_b(CL::SQ);
    const T inv = Ar<T>::rcp_f(sa + sb);   // as in roe_state
    // b1 = gm1 ic^2; c = c2 ic (= sqrt c2); ic = c2^-1/2; c2 = gm1 (H - hq2)
    rb.ic = fmaT(rb.b1 * gm1, r.ic + r.ic, rb.ic);
    const T ic3 = r.ic * r.ic * r.ic;
    const T c2b = halve(fmaT(rb.c, r.ic, -rb.ic * ic3));
    rb.H += c2b * gm1;
    rb.hq2 -= c2b * gm1;
    T invb = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const T ub = rb.u[k] + r.u[k] * rb.hq2;
        gab[k] += ub * inv;
        gbb[k] += ub * inv;
        invb += ub * (get_a(CL::SU + k) + get_b(CL::SU + k));
    }
    gab[DIM] += rb.H * inv;
    gbb[DIM] += rb.H * inv;
    invb += rb.H * (get_a(CL::SH) + get_b(CL::SH));
    const T sb_ = -invb * inv * inv;
    gab[DIM + 1] += sb_ + rb.rt * sb;
    gbb[DIM + 1] += sb_ + rb.rt * sa;
}

// adjoint of the reconstruction: fb -> bars of a..e (accumulated) and of lam
template <typename T>
__device__ __forceinline__ void recon_adj(T a, T b, T c, T d, T e, T lam, T eps, T fb, T* xb, T& lamb)
{
    const T q0 = T(0.5) * (c + d);
    const T q1 = fmaT(T(1.5), c, T(-0.5) * b);
    const T q2 = fmaT(T(1.0 / 3.0), c, fmaT(T(5.0 / 6.0), d, T(-1.0 / 6.0) * e));
    const T q3 = fmaT(T(1.0 / 3.0), a, fmaT(T(-7.0 / 6.0), b, T(11.0 / 6.0) * c));
    const T b0 = (d - c) * (d - c), b1 = (c - b) * (c - b);
    const T t2 = fmaT(T(-2), d, c) + e, s2 = fmaT(T(-4), d, T(3) * c) + e;
    const T be2 = fmaT(T(13.0 / 12.0), t2 * t2, T(0.25) * (s2 * s2));
    const T t3 = fmaT(T(-2), b, a) + c, s3 = fmaT(T(-4), b, a) + T(3) * c;
    const T be3 = fmaT(T(13.0 / 12.0), t3 * t3, T(0.25) * (s3 * s3));
    const T tt = fmaT(T(-4), b + d, a + e) + T(6) * c, st = fmaT(T(2), b - d, e - a);
    const T tau = fmaT(T(13.0 / 12.0), tt * tt, T(0.25) * (st * st));
    const T te = fmaT(T(-2), c, b + d);
    const T E = (te * te) * T(1.0 / 45.0);
    const T dk[4] = {T(0.4), T(0.2), T(0.3), T(0.1)};
    const T beta[4] = {b0, b1, be2, be3};
    const T lt = lam * tau;
    T D[4], al[4];
    T S = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        D[k] = fmaT(lam, beta[k], (k < 2 ? E : T(0)) + eps);
        al[k] = dk[k] * (T(1) + lt / D[k]);
        S += al[k];
    }
    const T iS = T(1) / S;
    const T q[4] = {q0, q1, q2, q3};
    T fh = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) fh = fmaT(al[k] * iS, q[k], fh);
    // reverse
    T qb[4], ltb = T(0), betab[4], Eb = T(0);
    lamb = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        qb[k] = fb * al[k] * iS;
        const T alb = (q[k] - fh) * fb * iS;
        const T r = alb * dk[k] / D[k];
        ltb += r;
        const T Db = -r * (lt / D[k]);
        lamb += Db * beta[k];
        betab[k] = Db * lam;
        if (k < 2) Eb += Db;
    }
    lamb += ltb * tau;
    const T taub = ltb * lam;
    T ab = T(0), bb = T(0), cb = T(0), db = T(0), eb = T(0);
    // beta_0, beta_1
    db += T(2) * (d - c) * betab[0]; cb -= T(2) * (d - c) * betab[0];
    cb += T(2) * (c - b) * betab[1]; bb -= T(2) * (c - b) * betab[1];
    // beta_2
    T tb = betab[2] * T(13.0 / 6.0) * t2, sb = betab[2] * T(0.5) * s2;
    cb += tb + T(3) * sb; db += T(-2) * tb - T(4) * sb; eb += tb + sb;
    // beta_3
    tb = betab[3] * T(13.0 / 6.0) * t3; sb = betab[3] * T(0.5) * s3;
    ab += tb + sb; bb += T(-2) * tb - T(4) * sb; cb += tb + T(3) * sb;
    // tau_5
    tb = taub * T(13.0 / 6.0) * tt; sb = taub * T(0.5) * st;
    ab += tb - sb; eb += tb + sb; bb += T(-4) * tb + T(2) * sb; db += T(-4) * tb - T(2) * sb; cb += T(6) * tb;
    // E
    tb = Eb * T(2.0 / 45.0) * te;
    bb += tb; cb -= T(2) * tb; db += tb;
    // candidate fluxes
    ab += qb[3] * T(1.0 / 3.0);
    bb += T(-0.5) * qb[1] + T(-7.0 / 6.0) * qb[3];
    cb += T(0.5) * qb[0] + T(1.5) * qb[1] + T(1.0 / 3.0) * qb[2] + T(11.0 / 6.0) * qb[3];
    db += T(0.5) * qb[0] + T(5.0 / 6.0) * qb[2];
    eb += T(-1.0 / 6.0) * qb[2];
    xb[0] += ab; xb[1] += bb; xb[2] += cb; xb[3] += db; xb[4] += eb;
}

struct VjpArgs {
    const void* U;      // state, interior only (the caller's array)
    const void* W;      // cotangent, interior only
    void* G;            // gradient, interior only (written / accumulated)
    void* ghost;        // [line][6][NV] gradients of ghost cells
    int* n_weno_tiles;  // tiles of this direction with a WENO face (zero before pass 0)
    int* weno_tiles;    // their linear tile indices, in no particular order (pass 0 appends)
    int tiles[3];       // tile grid of this direction (set by the launcher)
    int accumulate;     // 0: G = ..., 1: G += ... (pass 0; pass 1 always adds)
    int n[3];
    long long sy, sz, sv, off0;
    double inv_dx, eps_h, gamma, eps, c_lambda;
    double slim;   // 60 sqrt(eps_h), as in the forward sweep
    int hybrid;
    // boundary conditions of this direction, for the ghost cells computed
    // while staging (the fields stage_cell reads: bc_lo, bc_hi, bc_state,
    // lo0, dx0, lo1, dx1, tm = null, xs_fixed)
    SweepArgs bc;
    // cell primitives (cell_prims, PrimLayout records at STRIDE g): P read
    // (an earlier direction stored them), Pout computed and stored for the
    // tile's own cells, both null: computed and kept to the tile (FP64 only)
    const void* P;
    void* Pout;
};

// A tile is LINES grid lines x SEG cells along the sweep, one thread per
// face.  Lines along x take one line of 59 cells.  For y and z lines in FP32
// a tile takes 8 x-adjacent lines of 27 cells, so that the strided loads of
// one line position cover a 32-byte sector; in FP64 the arithmetic bounds
// those sweeps and one line per tile keeps 4 CTAs per SM resident.
template <typename T, int DIM, int DIR> struct VjpTile {
    static constexpr int LINES = (DIR != 0 && sizeof(T) == 4) ? 8 : 1;
    static constexpr int SEG = LINES == 1 ? 59 : 27;
    static constexpr int NT = LINES * (SEG + 5);
};

template <typename T, int DIM, int DIR, int PASS>
struct VjpSmem {
    static constexpr int LINES = VjpTile<T, DIM, DIR>::LINES;
    static constexpr int SEG = VjpTile<T, DIM, DIR>::SEG;
    static constexpr int NF = SEG + 5;          // faces c0-2 .. c0+SEG+2 per line
    static constexpr int NC = SEG + 10;         // cells c0-5 .. c0+SEG+4 per line
    static constexpr int LNF = LINES * NF, LNC = LINES * NC;
    static constexpr int NQ = CellLayout<DIM>::NQ;
    static constexpr int NV = DIM + 2;
    // per face: U and F bars of the six stencil cells (pass 1) or the two
    // bar vectors of a linear-upwind face (pass 0, NUF entries), Roe-field
    // bars of cells 2 and 3 (the face's neighbours), the three LLF speed
    // bars, and (as one int) the stencil slots of the cells attaining the
    // speeds and whether the pass takes the face
    // per cell after the record: 1/sqrt(rho), 1/c and, in FP64, p and c
    // (in FP32 the per-cell reverse recomputes those two: two more staged
    // rows cost the shared-memory-bound float tiles more than they save)
    static constexpr int NX = sizeof(T) == 8 ? 4 : 2;
    static constexpr int NUF = 2 * NV;
    static constexpr int NUFF = PASS == 0 ? NUF : 6 * NUF;
    static constexpr int NRB = DIM + 2;
    static constexpr int NFB = NUFF + 2 * NRB + 3;
    static constexpr size_t bytes =
        sizeof(T) * ((size_t)(NQ + NX) * LNC + (size_t)NV * LNC + (size_t)LNF * NFB) + sizeof(int) * (size_t)LNF;
};

// Residency of the WENO pass: its per-face reverse needs more than 255
// registers, which leaves 8 warps per SM in FP64.  FP32 code needs more
// warps to hide its latencies, so its register count is capped at 128 (8
// CTAs of the 64-thread x tiles, 2 of the 256-thread y/z tiles) at the cost
// of spills.
template <typename T, int NT, int PASS> struct VjpMinBlocks {
    static constexpr int value = PASS == 0 ? 1 : (sizeof(T) == 4 ? (NT == 64 ? 8 : 2) : 1);
};

// One tile of one direction of the VJP: tile (bx, by, bz) = LINES grid lines
// x SEG cells; shared arrays hold position p of line l at p * LINES + l.
// Returns (to every thread, pass 0) whether a face of the tile took WENO.
template <typename T, int DIM, int DIR, int PASS>
__device__ __forceinline__ bool vjp_tile(const VjpArgs& a, int bx, int by, int bz, unsigned char* smem_raw)
{
    using CL = CellLayout<DIM>;
    using SM = VjpSmem<T, DIM, DIR, PASS>;
    constexpr int NV = DIM + 2, NQ = CL::NQ, SEG = SM::SEG, NF = SM::NF;
    constexpr int LINES = SM::LINES, LNF = SM::LNF, LNC = SM::LNC;
    constexpr int NT = VjpTile<T, DIM, DIR>::NT;
    constexpr int NUF = SM::NUF, NUFF = SM::NUFF, NRB = SM::NRB;
    T* cq = reinterpret_cast<T*>(smem_raw);   // [NQ + NX][NC][LINES] records, 1/sqrt(rho), 1/c (, p, c)
    T* wq = cq + (NQ + SM::NX) * LNC;         // [NV][NC][LINES] cotangent
    T* UF = wq + NV * LNC;                    // [NF][LINES][NUFF] U and F bars (see below)
    T* RB = UF + LNF * NUFF;                  // [NF][LINES][2][NRB] Roe-field bars of cells 2 and 3
    T* SP = RB + LNF * 2 * NRB;               // [NF][LINES][3] LLF speed bars
    int* SL = reinterpret_cast<int*>(SP + LNF * 3);   // [NF][LINES] slots attaining the speeds, face taken
    constexpr int SKIP = 1 << 12;   // the face belongs to the other pass

    const int nd = a.n[DIR];
    const int c0 = bx * SEG;
    // line coordinates: the two indices other than DIR; the lines of a
    // multi-line tile are consecutive in x
    int ix0 = 0, j = 0, k = 0;
    if (DIR == 0) { j = by; k = bz; }
    else if (DIR == 1) { ix0 = by * LINES; k = bz; }
    else { ix0 = by * LINES; j = bz; }
    const int nlx = DIR == 0 ? 1 : (a.n[0] - ix0 < LINES ? a.n[0] - ix0 : LINES);   // lines present
    const long long sd = DIR == 0 ? 1LL : (DIR == 1 ? a.sy : a.sz);
    const long long base0 = a.off0 + (long long)ix0 + (long long)j * a.sy + (long long)k * a.sz;
    const T* Ug = reinterpret_cast<const T*>(a.U);
    const T* Wg = reinterpret_cast<const T*>(a.W);
    const T gamma = T(a.gamma);

    // stage cells c0-5 .. c0+SEG+4 that exist (-3 .. nd+2); ghost cells come
    // from the boundary conditions, and the cotangent is zero on them
    for (int idx = threadIdx.x; idx < LNC; idx += NT) {
        const int p = idx / LINES, l = idx - (idx / LINES) * LINES;
        const int cell = c0 - 5 + p;
        if (l < nlx && cell >= -3 && cell <= nd + 2) {
            // in-plane index of the line for the boundary conditions: the row
            // for x sweeps, the column for y and z sweeps
            const int line = DIR == 0 ? j : ix0 + l;
            using PL = PrimLayout<DIM>;
            T U[NV], q[NQ], inv[2], P[PL::NP];
            if constexpr (sizeof(T) == 8) {
                long long gs = 0;
                bool flip = false;
                const int fixed = cell_source<DIR>(a.bc, base0 + l, line, cell, nd, gs, flip);
                if (fixed >= 0) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) U[v] = a.bc.bc_state[fixed][v];
                    cell_prims<T, DIM>(U, gamma, gamma - T(1), P, inv);
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v) U[v] = Ug[gs + v * a.sv];
                    if (a.P != nullptr) {
                        // 1/sqrt(rho) = sqrt(rho) / rho and 1/c from the
                        // stored record (within an ulp or two of the staged
                        // values)
                        load_prims<DIM>(reinterpret_cast<const T*>(a.P), gs, P);
                        inv[0] = P[PL::SQ] * P[PL::IRHO];
                        inv[1] = Ar<T>::rcp_f(P[PL::C]);
                    } else {
                        cell_prims<T, DIM>(U, gamma, gamma - T(1), P, inv);
                        if (a.Pout != nullptr && cell >= c0 && cell < c0 + SEG && cell < nd)
                            store_prims<DIM>(reinterpret_cast<T*>(a.Pout), gs, P);
                    }
                    if (flip) {
                        U[1 + DIR] = -U[1 + DIR];
                        P[PL::SU + DIR] = -P[PL::SU + DIR];
                    }
                }
            } else {
                // float: no stored primitives (the float tiles were measured
                // slower with the source lookup above)
                stage_cell<T, DIM, DIR>(a.bc, Ug, base0 + l, line, cell, nd, U);
                cell_prims<T, DIM>(U, gamma, gamma - T(1), P, inv);
            }
            const bool inside = cell >= 0 && cell < nd;
            const long long g = base0 + l + (long long)cell * sd;
#pragma unroll
            for (int v = 0; v < NV; ++v) wq[v * LNC + idx] = inside ? Wg[g + v * a.sv] : T(0);
            cell_record<T, DIM, DIR>(U, P, q);
#pragma unroll
            for (int kk = 0; kk < NQ; ++kk) cq[kk * LNC + idx] = q[kk];
            cq[NQ * LNC + idx] = inv[0];
            cq[(NQ + 1) * LNC + idx] = inv[1];
            if constexpr (SM::NX == 4) {
                cq[(NQ + 2) * LNC + idx] = P[PrimLayout<DIM>::P];
                cq[(NQ + 3) * LNC + idx] = P[PrimLayout<DIM>::C];
            }
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) wq[v * LNC + idx] = T(0);
        }
    }
    __syncthreads();

    // ---- per face: forward recompute and reverse -------------------------
    const T slim = T(a.slim);
    const T lam_k = T(a.c_lambda / 3600.0);
    const T eps = T(a.eps), inv_dx = T(a.inv_dx);
    bool has_weno = false;
    for (int ff = threadIdx.x; ff < LNF; ff += NT) {
        const int f = ff / LINES, l = ff - (ff / LINES) * LINES;
        const int face = c0 - 2 + f;            // face i' between cells i'-1 and i'
        if (l >= nlx || face < 0 || face > nd) continue;
        // stencil cell j-2 = face-3 sits at position f of line l
        auto rec = [&](int m, int kk) -> T { return cq[kk * LNC + (f + m) * LINES + l]; };
        // pass 1 (WENO faces): U and F bars of each of the six stencil
        // cells; pass 0 (linear-upwind faces): the bars of the detector
        // difference (U slots) and of the central-flux sum (F slots)
        T* UFf = UF + (size_t)ff * NUFF;
        T* RBf = RB + (size_t)ff * 2 * NRB;    // Roe-field bars of cells 2 and 3
        // cotangent of the face flux: (w_{right} - w_{left}) / dx
        T phi[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v)
            phi[v] = (wq[v * LNC + (f + 3) * LINES + l] - wq[v * LNC + (f + 2) * LINES + l]) * inv_dx;

        auto ga = [&](int kk) -> T { return rec(2, kk); };
        auto gb = [&](int kk) -> T { return rec(3, kk); };
        const Roe<T, DIM> r = roe_state<T, DIM>(ga, gb, gamma - T(1));
        RoeBar<T, DIM> rb;
        zero(rb);
        T dU[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int kk = CL::U + v;
            dU[v] = fmaT(T(10), rec(2, kk) - rec(3, kk), fmaT(T(5), rec(4, kk) - rec(1, kk), rec(0, kk) - rec(5, kk)));
        }
        T w[NV];
        proj_all<T, DIM, DIR>(r, dU, w);
        const T lim = slim * r.rt;
        bool smooth = a.hybrid != 0;
#pragma unroll
        for (int s = 0; s < NV; ++s) smooth = smooth && abs_lt(w[s], lim);
        if (smooth != (PASS == 0)) {   // the other pass takes this face
            has_weno = has_weno || !smooth;
            SL[ff] = SKIP;
            continue;
        }
        // LLF speeds and the cells attaining them
        T am = rec(0, CL::LM), a0 = rec(0, CL::L0), ap = rec(0, CL::LP);
        int im = 0, i0 = 0, ip = 0;
#pragma unroll
        for (int m = 1; m < 6; ++m) {
            // the speeds are non-negative: compared on their bit patterns
            // (integer pipes), first index on ties as before
            const T xm = rec(m, CL::LM), x0 = rec(m, CL::L0), xp = rec(m, CL::LP);
            if (lt_nn(am, xm)) { am = xm; im = m; }
            if (lt_nn(a0, x0)) { a0 = x0; i0 = m; }
            if (lt_nn(ap, xp)) { ap = xp; ip = m; }
        }
        T alb_m = T(0), alb_0 = T(0), alb_p = T(0);
        T wb[NV], dUb[NV];
#pragma unroll
        for (int s = 0; s < NV; ++s) { wb[s] = T(0); dUb[s] = T(0); }
        if constexpr (PASS == 0) {
            // F = [central(F) + a0 dU + k0 R^{u-c} + k3 R^{u+c}] / 60 with
            // k0 = (am - a0) w_0, k3 = (ap - a0) w_last, the form the forward
            // sweep evaluates (ups_dissipation_add); the gather applies the
            // central weights to the bar Fb of the sum
            T Fb[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                Fb[v] = phi[v] * T(1.0 / 60.0);
                UFf[CL::F + v] = Fb[v];
            }
            constexpr int LAST = NV - 1;
            const T k0 = (am - a0) * w[0], k3 = (ap - a0) * w[LAST];
            const T sum = k0 + k3, dd = k3 - k0;
            const T unc = r.u[DIR] * r.c;
            // out[0] += s; out[1 + k] += u_k s (+ c dd along DIR); out[E] += H s + u_n c dd
            T sb = fmaT(r.H, Fb[LAST], Fb[0]);
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                sb = fmaT(r.u[k], Fb[1 + k], sb);
                rb.u[k] = fmaT(sum, Fb[1 + k], rb.u[k]);
            }
            const T ddb = fmaT(r.c, Fb[1 + DIR], unc * Fb[LAST]);
            rb.H = fmaT(sum, Fb[LAST], rb.H);
            const T uncb = dd * Fb[LAST];
            rb.u[DIR] = fmaT(uncb, r.c, rb.u[DIR]);
            rb.c = fmaT(uncb, r.u[DIR], fmaT(dd, Fb[1 + DIR], rb.c));
            const T k0b = sb - ddb, k3b = sb + ddb;
            alb_m = k0b * w[0];
            alb_p = k3b * w[LAST];
            wb[0] = k0b * (am - a0);
            wb[LAST] = k3b * (ap - a0);
            // a0 dU: the entropy and shear fields' speed
            T dot = T(0);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                dot = fmaT(Fb[v], dU[v], dot);
                dUb[v] = a0 * Fb[v];
            }
            alb_0 = dot - alb_m - alb_p;
        } else {
            // projections of the six cells, all fields
            T vv[6][NV], gg[6][NV];
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                T xu[NV], xf[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) { xu[v] = rec(m, CL::U + v); xf[v] = rec(m, CL::F + v); }
                proj_all<T, DIM, DIR>(r, xu, vv[m]);
                proj_all<T, DIM, DIR>(r, xf, gg[m]);
            }
            const T irt2 = T(1) / (r.rt * r.rt);
            T wch[NV];
            T lam[NV];
#pragma unroll
            for (int s = 0; s < NV; ++s) {
                const T al = s == 0 ? am : (s == NV - 1 ? ap : a0);
                lam[s] = lam_k * (w[s] * w[s]) * irt2;
                T fp[6], fm[6];
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    const T h = T(0.5) * gg[m][s], kq = T(0.5) * al * vv[m][s];
                    fp[m] = h + kq;
                    fm[m] = h - kq;
                }
                wch[s] = recon<T>(fp[0], fp[1], fp[2], fp[3], fp[4], lam[s], eps) +
                         recon<T>(fm[5], fm[4], fm[3], fm[2], fm[1], lam[s], eps);
            }
            T wchb[NV];
            back_proj_adj<T, DIM, DIR>(r, wch, phi, wchb, rb);
            T vb[6][NV], gbar[6][NV];
#pragma unroll
            for (int m = 0; m < 6; ++m)
#pragma unroll
                for (int s = 0; s < NV; ++s) { vb[m][s] = T(0); gbar[m][s] = T(0); }
#pragma unroll
            for (int s = 0; s < NV; ++s) {
                const T al = s == 0 ? am : (s == NV - 1 ? ap : a0);
                T fp[6], fm[6];
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    const T h = T(0.5) * gg[m][s], kq = T(0.5) * al * vv[m][s];
                    fp[m] = h + kq;
                    fm[m] = h - kq;
                }
                T xp[5] = {T(0), T(0), T(0), T(0), T(0)}, xm[5] = {T(0), T(0), T(0), T(0), T(0)};
                T lbp, lbm;
                recon_adj<T>(fp[0], fp[1], fp[2], fp[3], fp[4], lam[s], eps, wchb[s], xp, lbp);
                recon_adj<T>(fm[5], fm[4], fm[3], fm[2], fm[1], lam[s], eps, wchb[s], xm, lbm);
                // fm input order was m = 5, 4, 3, 2, 1
                T fpb[6] = {xp[0], xp[1], xp[2], xp[3], xp[4], T(0)};
                T fmb[6] = {T(0), xm[4], xm[3], xm[2], xm[1], xm[0]};
                T alb = T(0);
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    gbar[m][s] += T(0.5) * (fpb[m] + fmb[m]);
                    vb[m][s] += T(0.5) * al * (fpb[m] - fmb[m]);
                    alb += T(0.5) * vv[m][s] * (fpb[m] - fmb[m]);
                }
                if (s == 0) alb_m += alb;
                else if (s == NV - 1) alb_p += alb;
                else alb_0 += alb;
                // lam = c w^2 / (3600 rt^2)
                const T lb = lbp + lbm;
                wb[s] += lb * T(2) * lam_k * w[s] * irt2;
                rb.rt += lb * (T(-2) * lam[s] / r.rt);
            }
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                T xu[NV], xf[NV], xub[NV], xfb[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    xu[v] = rec(m, CL::U + v); xf[v] = rec(m, CL::F + v);
                    xub[v] = T(0); xfb[v] = T(0);
                }
                proj_all_adj<T, DIM, DIR>(r, xu, vb[m], xub, rb);
                proj_all_adj<T, DIM, DIR>(r, xf, gbar[m], xfb, rb);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    UFf[m * NUF + CL::U + v] = xub[v];
                    UFf[m * NUF + CL::F + v] = xfb[v];
                }
            }
        }
        // detector: w = L dU, dU = (U0 - U5) + 5 (U4 - U1) + 10 (U2 - U3)
        proj_all_adj<T, DIM, DIR>(r, dU, wb, dUb, rb);
        if constexpr (PASS == 0) {
#pragma unroll
            for (int v = 0; v < NV; ++v) UFf[CL::U + v] = dUb[v];
        } else {
            const T cd[6] = {T(1), T(-5), T(10), T(-10), T(5), T(-1)};
#pragma unroll
            for (int m = 0; m < 6; ++m)
#pragma unroll
                for (int v = 0; v < NV; ++v) UFf[m * NUF + CL::U + v] += cd[m] * dUb[v];
        }
        SP[ff * 3 + 0] = alb_m;
        SP[ff * 3 + 1] = alb_0;
        SP[ff * 3 + 2] = alb_p;
        SL[ff] = im | (i0 << 4) | (ip << 8);
#pragma unroll
        for (int kk = 0; kk < 2 * NRB; ++kk) RBf[kk] = T(0);
        roe_adj<T, DIM>(ga, gb, gamma, r, rb, RBf, RBf + NRB);
    }
    const bool any_weno = __syncthreads_or(has_weno ? 1 : 0) != 0;

    // ---- gather per cell: faces i' in [i-2, i+3], stencil slot m = i - i' + 3
    T* Gg = reinterpret_cast<T*>(a.G);
    T* ghost = reinterpret_cast<T*>(a.ghost);
    const bool first = c0 == 0, last = c0 + SEG >= nd;
    for (int idx = threadIdx.x; idx < LINES * (SEG + 6); idx += NT) {
        const int p = idx / LINES, l = idx - (idx / LINES) * LINES;
        const int cell = c0 - 3 + p;   // owned cells c0..c0+SEG-1 and boundary ghosts
        const bool owned = cell >= c0 && cell < c0 + SEG && cell < nd;
        const bool gl = first && cell < 0 && cell >= -3;
        const bool gr = last && cell >= nd && cell <= nd + 2;
        if (l >= nlx || (!owned && !gl && !gr)) continue;
        T qb[NQ];
#pragma unroll
        for (int kk = 0; kk < NQ; ++kk) qb[kk] = T(0);
        bool touched = false;
        // pass 0 in FP64: the face (index into the face arrays) that gives
        // this cell its stencil slot m, -1 where none does
        int fslot[6] = {-1, -1, -1, -1, -1, -1};
        // central-flux and detector weights of stencil slot m (pass 0 in FP32)
        constexpr T cf[6] = {T(1), T(-8), T(37), T(37), T(-8), T(1)};
        constexpr T cd[6] = {T(1), T(-5), T(10), T(-10), T(5), T(-1)};
#pragma unroll
        for (int m = 5; m >= 0; --m) {
            const int fi = cell - m + 3;   // faces in increasing order
            if (fi < 0 || fi > nd) continue;
            const int f = fi - (c0 - 2);
            if (f < 0 || f >= NF) continue;
            const int ff = f * LINES + l;
            const int sl = SL[ff];
            if (sl & SKIP) continue;
            touched = true;
            // the entries this cell receives from face fi, in the record
            // layout; the others are zero for it
            if constexpr (PASS == 1) {
                const T* uf = UF + (size_t)ff * NUFF + m * NUF;
#pragma unroll
                for (int kk = 0; kk < NUF; ++kk) qb[kk] += uf[kk];
            } else if constexpr (sizeof(T) == 8) {
                fslot[m] = ff;
            } else {
                const T* uf = UF + (size_t)ff * NUFF;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    qb[CL::U + v] = fmaT(cd[m], uf[CL::U + v], qb[CL::U + v]);
                    qb[CL::F + v] = fmaT(cf[m], uf[CL::F + v], qb[CL::F + v]);
                }
            }
            if (m == 2 || m == 3) {
                const T* rbp = RB + ((size_t)ff * 2 + (m - 2)) * NRB;
#pragma unroll
                for (int kk = 0; kk < NRB; ++kk) qb[CL::SU + kk] += rbp[kk];
            }
            if ((sl & 15) == m) qb[CL::LM] += SP[ff * 3 + 0];
            if (((sl >> 4) & 15) == m) qb[CL::L0] += SP[ff * 3 + 1];
            if (((sl >> 8) & 15) == m) qb[CL::LP] += SP[ff * 3 + 2];
        }
        if constexpr (PASS == 0 && sizeof(T) == 8) {
            // stencil weights of slot m: detector (1, -5, 10, -10, 5, -1)
            // on the U slots, central flux (1, -8, 37, 37, -8, 1) on the F
            // slots, applied as sums and differences of the symmetric pairs
            // (10 FP64 operations per variable instead of 12; in FP32 the
            // six loads held at once cost the 256-thread tiles a CTA per SM,
            // so FP32 keeps one multiply-add per slot)
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                T bu[6], bf[6];
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    const T* uf = UF + (size_t)(fslot[m] < 0 ? 0 : fslot[m]) * NUFF;
                    bu[m] = fslot[m] < 0 ? T(0) : uf[CL::U + v];
                    bf[m] = fslot[m] < 0 ? T(0) : uf[CL::F + v];
                }
                qb[CL::U + v] = fmaT(T(10), bu[2] - bu[3], fmaT(T(5), bu[4] - bu[1], bu[0] - bu[5]));
                qb[CL::F + v] = fmaT(T(37), bf[2] + bf[3], fmaT(T(-8), bf[1] + bf[4], bf[0] + bf[5]));
            }
        }
        if (PASS == 1 && !touched) continue;
        const int pc = cell - (c0 - 5);
        T U[NV], Ub[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = cq[(CL::U + v) * LNC + pc * LINES + l];
        const int ci = pc * LINES + l;
        const T isq = cq[NQ * LNC + ci], ic = cq[(NQ + 1) * LNC + ci];
        T pc_p, pc_c;
        if constexpr (SM::NX == 4) {
            pc_p = cq[(NQ + 2) * LNC + ci];
            pc_c = cq[(NQ + 3) * LNC + ci];
        } else {
            // p and c as cell_prims forms them
            const T irho = isq * isq;
            T m2 = T(0);
#pragma unroll
            for (int k = 0; k < DIM; ++k) m2 = fmaT(U[1 + k], U[1 + k], m2);
            pc_p = (gamma - T(1)) * fmaT(T(-0.5) * irho, m2, U[DIM + 1]);
            pc_c = gamma * pc_p * irho * ic;
        }
        cell_adj<T, DIM, DIR>(U, gamma, isq, ic, pc_p, pc_c, qb, Ub);
        if (owned) {
            const long long g = base0 + l + (long long)cell * sd;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if (PASS == 1 || a.accumulate) Gg[g + v * a.sv] += Ub[v];
                else Gg[g + v * a.sv] = Ub[v];
            }
        } else {
            const long long i = ix0 + l;
            const long long line = DIR == 0 ? ((long long)k * a.n[1] + j)
                                            : (DIR == 1 ? ((long long)k * a.n[0] + i) : ((long long)j * a.n[0] + i));
            const int slot = gl ? (-cell - 1) : (3 + cell - nd);   // 0..2 left (-1,-2,-3), 3..5 right
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if (PASS == 1) ghost[(line * 6 + slot) * NV + v] += Ub[v];
                else ghost[(line * 6 + slot) * NV + v] = Ub[v];
            }
        }
    }
    return any_weno;
}

// Pass 0: one CTA per tile; a tile with a WENO face appends its index to
// the list.  Pass 1: a grid of resident CTAs takes the listed tiles in turn
// (each tile writes only its own cells and ghost slots, so the order in
// which the tiles are taken does not change the result).
template <typename T, int DIM, int DIR, int PASS>
__global__ void __launch_bounds__(VjpTile<T, DIM, DIR>::NT, VjpMinBlocks<T, VjpTile<T, DIM, DIR>::NT, PASS>::value)
    k_vjp(VjpArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if constexpr (PASS == 0) {
        const bool any = vjp_tile<T, DIM, DIR, 0>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem_raw);
        if (any && threadIdx.x == 0)
            a.weno_tiles[atomicAdd(a.n_weno_tiles, 1)] = blockIdx.x + a.tiles[0] * (blockIdx.y + a.tiles[1] * blockIdx.z);
    } else {
        const int n = *a.n_weno_tiles;
        for (int it = blockIdx.x; it < n; it += gridDim.x) {
            const int t = a.weno_tiles[it];
            const int bx = t % a.tiles[0], byz = t / a.tiles[0];
            vjp_tile<T, DIM, DIR, 1>(a, bx, byz % a.tiles[1], byz / a.tiles[1], smem_raw);
            __syncthreads();   // shared memory is reused by the next tile
        }
    }
}

// ghost-cell gradients back to the interior cells they copy (the adjoint of
// the boundary conditions); fixed inflow states receive nothing
template <typename T, int DIM>
__global__ void k_ghost_adj(GhostArgs a, const void* ghost_, void* G_)
{
    constexpr int NV = DIM + 2;
    const int d = a.dir;
    const int nd = a.n[d];
    int e0, e1;
    if (d == 0) { e0 = a.n[1]; e1 = a.n[2]; }
    else if (d == 1) { e0 = a.n[0]; e1 = a.n[2]; }
    else { e0 = a.n[0]; e1 = a.n[1]; }
    const long long lines = (long long)e0 * e1;
    const long long sd = d == 0 ? 1LL : (d == 1 ? a.sy : a.sz);
    const T* ghost = reinterpret_cast<const T*>(ghost_);
    T* G = reinterpret_cast<T*>(G_);
    for (long long ln = blockIdx.x * (long long)blockDim.x + threadIdx.x; ln < lines;
         ln += (long long)gridDim.x * blockDim.x) {
        const int p0 = (int)(ln % e0), p1 = (int)(ln / e0);
        int i, j, k;
        if (d == 0) { i = 0; j = p0; k = p1; }
        else if (d == 1) { i = p0; j = 0; k = p1; }
        else { i = p0; j = p1; k = 0; }
        const long long base = a.off0 + (long long)i + (long long)j * a.sy + (long long)k * a.sz;
        for (int slot = 0; slot < 6; ++slot) {
            const int side = slot / 3, gl = slot % 3 + 1;
            int bc = side == 0 ? a.bc_lo : a.bc_hi;
            if (bc == BC_DMR_BOTTOM) {
                const double x = a.lo0 + (i + 0.5) * a.dx0;
                bc = x < 1.0 / 6.0 ? BC_INFLOW : BC_REFLECT;
            } else if (bc == BC_DMR_TOP || bc == BC_JET) {
                bc = BC_INFLOW;
            }
            if (bc == BC_INFLOW) continue;
            int src;
            if (bc == BC_TRANSMISSIVE) src = side == 0 ? 0 : nd - 1;
            else if (bc == BC_REFLECT) src = side == 0 ? gl - 1 : nd - gl;
            else src = side == 0 ? nd - gl : gl - 1;
            const long long g = base + (long long)src * sd;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                T val = ghost[(ln * 6 + slot) * NV + v];
                if (bc == BC_REFLECT && v == 1 + d) val = -val;
                G[g + v * a.sv] += val;
            }
        }
    }
}

}  // namespace wis
