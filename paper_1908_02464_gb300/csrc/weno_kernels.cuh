// Kernels of the regularized WENO-IS Euler solver (sm_103a).
//
//   k_sweep   one direction of the semi-discrete operator (Eq. goveq5): a
//             tile of LINES grid lines x SEG cells along the sweep, staged in
//             shared memory with a 3-cell halo; every face of the tile goes
//             through the detector (Eq. eq27-28) and either the optimal
//             linear upwind flux (Eq. linearupwind) or, after compaction
//             into a per-tile queue, the characteristic regularized WENO-IS
//             flux (Sec. 2.4, Eq. eq8-r); the tile then takes the flux
//             divergence and writes an accumulator, a right-hand side or the
//             RK3 stage combination (Sec. 4).
//   k_ghost   three ghost layers of one direction (boundary conditions).
//   k_cfl     CFL wave-speed max-reduction and admissibility check.
//   k_dt, k_post   single-thread time-step bookkeeping on the device.
//   k_totals  conserved totals, FP64 accumulation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "weno_device.cuh"

namespace wis {

// Device-resident time state of a context.
struct DevTime {
    double t;                       // time of the current state
    double dt;                      // step in progress (0: nothing to do)
    double t_end;                   // target of the step in progress
    unsigned long long smax_bits;   // max wave speed sum (bits of a positive double)
    long long steps;                // completed steps
    int status;                     // 0 ok, else WENO_ERR_NONPHYSICAL latched
    int clipped;                    // 1 if dt was clipped to reach t_end
};

enum { MODE_ACC_SET = 0, MODE_ACC_ADD = 1, MODE_COMBINE = 2, MODE_RHS = 3 };

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
    int hybrid;
};

template <typename T, int DIM>
struct FaceRec {
    // face record kept for queued WENO faces: Roe state, detector, speeds
    static constexpr int NV = DIM + 2;
    static constexpr int U = 0;               // u[DIM]
    static constexpr int C = DIM;
    static constexpr int IC = DIM + 1;
    static constexpr int H = DIM + 2;
    static constexpr int B1 = DIM + 3;
    static constexpr int HQ2 = DIM + 4;
    static constexpr int RT = DIM + 5;
    static constexpr int W = DIM + 6;         // dv[NV]
    static constexpr int AM = W + NV;         // alpha^{u-c}
    static constexpr int A0 = AM + 1;         // alpha^{u}, shear
    static constexpr int AP = AM + 2;         // alpha^{u+c}
    static constexpr int NR = AM + 3;
};

template <typename T, int DIM, int LINES, int SEG>
struct SweepSmem {
    static constexpr int CELLS = SEG + 6;
    static constexpr int FACES = SEG + 1;
    static constexpr int NCELL = LINES * CELLS;
    static constexpr int NFACE = LINES * FACES;
    static constexpr int NQ = CellLayout<DIM>::NQ;
    static constexpr int NV = DIM + 2;
    static constexpr int NR = FaceRec<T, DIM>::NR;
    static constexpr size_t bytes =
        sizeof(T) * ((size_t)NQ * NCELL + (size_t)NV * NFACE + (size_t)NR * NFACE) +
        sizeof(int) * (size_t)NFACE;
};

template <typename T, int DIM, int DIR, int LINES, int SEG, int NT, bool DET64>
__global__ void __launch_bounds__(NT) k_sweep(SweepArgs a)
{
    using CL = CellLayout<DIM>;
    using FR = FaceRec<T, DIM>;
    using SM = SweepSmem<T, DIM, LINES, SEG>;
    constexpr int NV = DIM + 2;
    constexpr int NQ = CL::NQ;
    constexpr int CELLS = SM::CELLS, FACES = SM::FACES;
    constexpr int NCELL = SM::NCELL, NFACE = SM::NFACE;
    constexpr int NR = FR::NR;

    if (a.tm != nullptr) {
        if (a.tm->status != 0 || !(a.tm->dt > 0.0)) return;
    }

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* cq = reinterpret_cast<T*>(smem_raw);     // [NQ][NCELL]
    T* fh = cq + NQ * NCELL;                    // [NV][NFACE]
    T* fr = fh + NV * NFACE;                    // [NR][NFACE]
    int* queue = reinterpret_cast<int*>(fr + NR * NFACE);
    __shared__ int qcount;
    __shared__ unsigned int wcount;

    int seg_blk, line0, pb;
    if (DIR == 0) { seg_blk = blockIdx.x; line0 = blockIdx.y * LINES; pb = blockIdx.z; }
    else if (DIR == 1) { seg_blk = blockIdx.y; line0 = blockIdx.x * LINES; pb = blockIdx.z; }
    else { seg_blk = blockIdx.z; line0 = blockIdx.x * LINES; pb = blockIdx.y; }
    const int nd = a.n[DIR];
    const int c0 = seg_blk * SEG;
    const int nline = (DIR == 0) ? a.n[1] : a.n[0];
    const long long sd = DIR == 0 ? 1LL : (DIR == 1 ? a.sy : a.sz);
    const long long sl = DIR == 0 ? a.sy : 1LL;
    const long long sp = DIR == 2 ? a.sy : a.sz;
    const T gamma = T(a.gamma);

    const T* Ug = reinterpret_cast<const T*>(a.U);

    if (threadIdx.x == 0) { qcount = 0; wcount = 0u; }

    // ---- stage the tile (cells c0-3 .. c0+SEG+2 of LINES lines) --------
    for (int idx = threadIdx.x; idx < NCELL; idx += NT) {
        int l, p;
        if (DIR == 0) { l = idx / CELLS; p = idx - l * CELLS; }
        else { p = idx / LINES; l = idx - p * LINES; }
        const int line = line0 + l;
        const int along = c0 - 3 + p;
        if (line < nline && along < nd + 3) {
            const long long g = a.off0 + (long long)line * sl + (long long)pb * sp + (long long)along * sd;
            T U[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) U[v] = Ug[g + v * a.sv];
            T q[NQ];
            cell_prepare<T, DIM, DIR>(U, gamma, q);
#pragma unroll
            for (int k = 0; k < NQ; ++k) cq[k * NCELL + idx] = q[k];
        }
    }
    __syncthreads();

    auto cidx = [](int l, int p) -> int { return DIR == 0 ? l * CELLS + p : p * LINES + l; };
    auto fdec = [](int f, int& l, int& p) {
        if (DIR == 0) { l = f / FACES; p = f - l * FACES; }
        else { p = f / LINES; l = f - p * LINES; }
    };

    const T eps_h = T(a.eps_h);
    const int lane = threadIdx.x & 31;
    unsigned int my_weno = 0;

    // ---- phase 1: detector, linear upwind faces, queue of WENO faces -----
    for (int f0 = 0; f0 < NFACE; f0 += NT) {
        const int f = f0 + threadIdx.x;
        int l = 0, p = 0;
        bool valid = f < NFACE;
        if (valid) {
            fdec(f, l, p);
            valid = (line0 + l < nline) && (c0 + p <= nd);
        }
        bool weno = false;
        if (valid) {
            auto ga = [&](int k) -> T { return cq[k * NCELL + cidx(l, p + 2)]; };
            auto gb = [&](int k) -> T { return cq[k * NCELL + cidx(l, p + 3)]; };
            const Roe<T, DIM> r = roe_state<T, DIM>(ga, gb, gamma);
            // Eq. eq28: dU = (U_{j-2} + 10 U_j + 5 U_{j+2}) - (5 U_{j-1} + 10 U_{j+1} + U_{j+3})
            T dU[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const int k = CL::U + v;
                if (DET64) {
                    const double u0 = (double)cq[k * NCELL + cidx(l, p + 0)];
                    const double u1 = (double)cq[k * NCELL + cidx(l, p + 1)];
                    const double u2 = (double)cq[k * NCELL + cidx(l, p + 2)];
                    const double u3 = (double)cq[k * NCELL + cidx(l, p + 3)];
                    const double u4 = (double)cq[k * NCELL + cidx(l, p + 4)];
                    const double u5 = (double)cq[k * NCELL + cidx(l, p + 5)];
                    dU[v] = (T)((u0 + fmaT(10.0, u2, 5.0 * u4)) - (u5 + fmaT(10.0, u3, 5.0 * u1)));
                } else {
                    const T u0 = cq[k * NCELL + cidx(l, p + 0)];
                    const T u1 = cq[k * NCELL + cidx(l, p + 1)];
                    const T u2 = cq[k * NCELL + cidx(l, p + 2)];
                    const T u3 = cq[k * NCELL + cidx(l, p + 3)];
                    const T u4 = cq[k * NCELL + cidx(l, p + 4)];
                    const T u5 = cq[k * NCELL + cidx(l, p + 5)];
                    dU[v] = (u0 + fmaT(T(10), u2, T(5) * u4)) - (u5 + fmaT(T(10), u3, T(5) * u1));
                }
            }
            T w[NV];
            proj_all<T, DIM, DIR>(r, dU, w);
            // sigma^s = (dv^s / rho~)^2 < eps_h  <=>  dv^2 < eps_h rho~^2
            const T lim = eps_h * (r.rt * r.rt);
            bool smooth = a.hybrid != 0;
#pragma unroll
            for (int s = 0; s < NV; ++s) {
                w[s] *= T(1.0 / 60.0);
                smooth = smooth && (w[s] * w[s] < lim);
            }
            // LLF speeds: max over the six stencil cells
            T am = cq[CL::LM * NCELL + cidx(l, p)];
            T a0 = cq[CL::L0 * NCELL + cidx(l, p)];
            T ap = cq[CL::LP * NCELL + cidx(l, p)];
#pragma unroll
            for (int m = 1; m < 6; ++m) {
                am = maxT(am, cq[CL::LM * NCELL + cidx(l, p + m)]);
                a0 = maxT(a0, cq[CL::L0 * NCELL + cidx(l, p + m)]);
                ap = maxT(ap, cq[CL::LP * NCELL + cidx(l, p + m)]);
            }
            if (smooth) {
                // Eq. linearupwind: central six-point flux plus sum_s R^s alpha^s dv^s
                T Fo[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const int k = CL::F + v;
                    const T f05 = cq[k * NCELL + cidx(l, p + 0)] + cq[k * NCELL + cidx(l, p + 5)];
                    const T f14 = cq[k * NCELL + cidx(l, p + 1)] + cq[k * NCELL + cidx(l, p + 4)];
                    const T f23 = cq[k * NCELL + cidx(l, p + 2)] + cq[k * NCELL + cidx(l, p + 3)];
                    Fo[v] = fmaT(T(37), f23, fmaT(T(-8), f14, f05)) * T(1.0 / 60.0);
                }
                T aw[NV];
                aw[0] = am * w[0];
#pragma unroll
                for (int s = 1; s < NV - 1; ++s) aw[s] = a0 * w[s];
                aw[NV - 1] = ap * w[NV - 1];
                back_proj_add<T, DIM, DIR>(r, aw, Fo);
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
                fr[FR::RT * NFACE + f] = r.rt;
#pragma unroll
                for (int s = 0; s < NV; ++s) fr[(FR::W + s) * NFACE + f] = w[s];
                fr[FR::AM * NFACE + f] = am;
                fr[FR::A0 * NFACE + f] = a0;
                fr[FR::AP * NFACE + f] = ap;
            }
            // a face is owned by the tile left of it, the last face by the last tile
            const int face = c0 + p;
            const bool owned = (p < SEG) || (face == nd);
            if (owned) {
                if (weno) ++my_weno;
                if (a.flags != nullptr) {
                    const int line = line0 + l;
                    long long fidx;
                    if (DIR == 0) fidx = ((long long)pb * a.n[1] + line) * (long long)(nd + 1) + face;
                    else if (DIR == 1) fidx = ((long long)pb * (nd + 1) + face) * (long long)a.n[0] + line;
                    else fidx = ((long long)face * a.n[1] + pb) * (long long)a.n[0] + line;
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
    const T eps = T(a.eps), clam = T(a.c_lambda);
    for (int qi = threadIdx.x; qi < nq; qi += NT) {
        const int f = queue[qi];
        int l, p;
        fdec(f, l, p);
        Roe<T, DIM> r;
#pragma unroll
        for (int k = 0; k < DIM; ++k) r.u[k] = fr[(FR::U + k) * NFACE + f];
        r.c = fr[FR::C * NFACE + f];
        r.ic = fr[FR::IC * NFACE + f];
        r.H = fr[FR::H * NFACE + f];
        r.b1 = fr[FR::B1 * NFACE + f];
        r.hq2 = fr[FR::HQ2 * NFACE + f];
        r.rt = fr[FR::RT * NFACE + f];
        const T irt = Ar<T>::rcp(r.rt);
        const T am = fr[FR::AM * NFACE + f];
        const T a0 = fr[FR::A0 * NFACE + f];
        const T ap = fr[FR::AP * NFACE + f];

        // shared parts of the projections (Eq. eqchara) of U_m and F_m, m = j-2..j+3
        T t1U[6], aU[6], t1F[6], aF[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const int ci = cidx(l, p + m);
            T xu[NV], xf[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                xu[v] = cq[(CL::U + v) * NCELL + ci];
                xf[v] = cq[(CL::F + v) * NCELL + ci];
            }
            T du = r.u[0] * xu[1], df = r.u[0] * xf[1];
#pragma unroll
            for (int k = 1; k < DIM; ++k) { du = fmaT(r.u[k], xu[1 + k], du); df = fmaT(r.u[k], xf[1 + k], df); }
            t1U[m] = r.b1 * (fmaT(r.hq2, xu[0], xu[DIM + 1]) - du);
            t1F[m] = r.b1 * (fmaT(r.hq2, xf[0], xf[DIM + 1]) - df);
            aU[m] = fmaT(r.u[DIR], xu[0], -xu[1 + DIR]) * r.ic;
            aF[m] = fmaT(r.u[DIR], xf[0], -xf[1 + DIR]) * r.ic;
        }

        T wch[NV];
#pragma unroll
        for (int s = 0; s < NV; ++s) {
            T vv[6], gg[6];
            T alpha;
            if (s == 0) {
                alpha = am;
#pragma unroll
                for (int m = 0; m < 6; ++m) { vv[m] = T(0.5) * (t1U[m] + aU[m]); gg[m] = T(0.5) * (t1F[m] + aF[m]); }
            } else if (s == 1) {
                alpha = a0;
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    const int ci = cidx(l, p + m);
                    vv[m] = cq[CL::U * NCELL + ci] - t1U[m];
                    gg[m] = cq[CL::F * NCELL + ci] - t1F[m];
                }
            } else if (s == NV - 1) {
                alpha = ap;
#pragma unroll
                for (int m = 0; m < 6; ++m) { vv[m] = T(0.5) * (t1U[m] - aU[m]); gg[m] = T(0.5) * (t1F[m] - aF[m]); }
            } else {
                // shear field s -> tangential direction t (skipping DIR)
                alpha = a0;
                int t = s - 2;
                if (t >= DIR) ++t;
                const T ut = r.u[t];
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    const int ci = cidx(l, p + m);
                    vv[m] = fmaT(-ut, cq[CL::U * NCELL + ci], cq[(CL::U + 1 + t) * NCELL + ci]);
                    gg[m] = fmaT(-ut, cq[CL::F * NCELL + ci], cq[(CL::F + 1 + t) * NCELL + ci]);
                }
            }
            // Eq. flxuspliting: f^{+-} = (g +- alpha v)/2
            T fp[6], fm[6];
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const T h = T(0.5) * gg[m];
                const T k = T(0.5) * alpha * vv[m];
                fp[m] = h + k;
                fm[m] = h - k;
            }
            // Eq. eq27, eq29: lambda = c (dv / rho~)^2
            const T dvr = fr[(FR::W + s) * NFACE + f] * irt;
            const T lam = clam * (dvr * dvr);
            // Eq. reconstruction: + on j-2..j+2, - on the mirrored j+3..j-1
            const T fplus = recon<T>(fp[0], fp[1], fp[2], fp[3], fp[4], lam, eps);
            const T fminus = recon<T>(fm[5], fm[4], fm[3], fm[2], fm[1], lam, eps);
            wch[s] = fplus + fminus;   // Eq. reconstruction1
        }
        T Fo[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) Fo[v] = T(0);
        back_proj_add<T, DIM, DIR>(r, wch, Fo);   // Eq. reconstruction2
#pragma unroll
        for (int v = 0; v < NV; ++v) fh[v * NFACE + f] = Fo[v];
    }
    __syncthreads();
    if (threadIdx.x == 0 && a.weno_count != nullptr && wcount != 0u)
        atomicAdd(a.weno_count, (unsigned long long)wcount);

    // ---- flux divergence and output ---------------------------------------
    const T inv_dx = T(a.inv_dx);
    T* outp = reinterpret_cast<T*>(a.out);
    T* accp = reinterpret_cast<T*>(a.acc);
    const T* Unp = reinterpret_cast<const T*>(a.Un);
    T dt = T(0), rka = T(a.rk_a), rkb = T(a.rk_b);
    if (a.mode == MODE_COMBINE) dt = T(a.tm->dt);
    bool bad = false;
    for (int idx = threadIdx.x; idx < LINES * SEG; idx += NT) {
        int l, p;
        if (DIR == 0) { l = idx / SEG; p = idx - l * SEG; }
        else { p = idx / LINES; l = idx - p * LINES; }
        const int line = line0 + l;
        const int cell = c0 + p;
        if (line >= nline || cell >= nd) continue;
        const long long g = a.off0 + (long long)line * sl + (long long)pb * sp + (long long)cell * sd;
        const int fl = DIR == 0 ? l * FACES + p : p * LINES + l;
        const int fr_ = DIR == 0 ? fl + 1 : fl + LINES;
        T rv[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) rv[v] = (fh[v * NFACE + fl] - fh[v * NFACE + fr_]) * inv_dx;
        if (a.mode == MODE_ACC_SET) {
#pragma unroll
            for (int v = 0; v < NV; ++v) accp[g + v * a.sv] = rv[v];
        } else if (a.mode == MODE_ACC_ADD) {
#pragma unroll
            for (int v = 0; v < NV; ++v) accp[g + v * a.sv] += rv[v];
        } else if (a.mode == MODE_RHS) {
#pragma unroll
            for (int v = 0; v < NV; ++v) outp[g + v * a.sv] = (accp ? accp[g + v * a.sv] : T(0)) + rv[v];
        } else {
            const int ci = cidx(l, p + 3);
            T nu[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                T tot = rv[v];
                if (accp) tot += accp[g + v * a.sv];
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
    if (bad) atomicOr(&a.tm->status, 1);
}

// ---------------------------------------------------------------- ghosts
struct GhostArgs {
    void* U;
    int dir;
    int n[3];
    long long sy, sz, sv, off0;
    int bc_lo, bc_hi;
    double bc_state[2][5];
    double lo0, dx0;     // x-axis geometry for the DMR boundaries
    DevTime* tm;         // stage time from tm (t + stage_c dt), or t_fixed
    double stage_c, t_fixed;
};

enum { BC_TRANSMISSIVE = 0, BC_REFLECT = 1, BC_PERIODIC = 2, BC_INFLOW = 3, BC_DMR_BOTTOM = 4,
       BC_DMR_TOP = 5 };

template <typename T, int DIM>
__global__ void k_ghost(GhostArgs a)
{
    constexpr int NV = DIM + 2;
    if (a.tm != nullptr && (a.tm->status != 0 || !(a.tm->dt > 0.0))) return;
    const int d = a.dir;
    const int nd = a.n[d];
    // perpendicular extents (i fastest where possible)
    int e0, e1;   // sizes of the two perpendicular index ranges
    if (d == 0) { e0 = a.n[1]; e1 = a.n[2]; }
    else if (d == 1) { e0 = a.n[0]; e1 = a.n[2]; }
    else { e0 = a.n[0]; e1 = a.n[1]; }
    const long long P = (long long)e0 * e1;
    const long long total = 2LL * 3LL * P;
    const long long sd = d == 0 ? 1LL : (d == 1 ? a.sy : a.sz);
    T* U = reinterpret_cast<T*>(a.U);
    double t = a.t_fixed;
    if (a.tm != nullptr) t = a.tm->t + a.stage_c * a.tm->dt;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
        const long long pp = id % P;
        const int gl = (int)((id / P) % 3) + 1;
        const int side = (int)(id / (3 * P));
        const int p0 = (int)(pp % e0), p1 = (int)(pp / e0);
        int i, j, k;
        if (d == 0) { i = 0; j = p0; k = p1; }
        else if (d == 1) { i = p0; j = 0; k = p1; }
        else { i = p0; j = p1; k = 0; }
        // address of the line's cell 0 along d (the along-d index is zero here)
        const long long base = a.off0 + (long long)i + (long long)j * a.sy + (long long)k * a.sz;
        const int dst = side == 0 ? -gl : nd - 1 + gl;
        int bc = side == 0 ? a.bc_lo : a.bc_hi;
        const double* fixed = nullptr;
        if (bc == BC_DMR_BOTTOM) {
            const double x = a.lo0 + (i + 0.5) * a.dx0;
            if (x < 1.0 / 6.0) { bc = BC_INFLOW; fixed = a.bc_state[0]; }
            else bc = BC_REFLECT;
        } else if (bc == BC_DMR_TOP) {
            const double x = a.lo0 + (i + 0.5) * a.dx0;
            const double xs = 1.0 / 6.0 + (1.0 + 20.0 * t) / sqrt(3.0);
            fixed = (x < xs) ? a.bc_state[0] : a.bc_state[1];
            bc = BC_INFLOW;
        } else if (bc == BC_INFLOW) {
            fixed = a.bc_state[0];
        }
        const long long gdst = base + (long long)dst * sd;
        if (bc == BC_INFLOW) {
#pragma unroll
            for (int v = 0; v < NV; ++v) U[gdst + v * a.sv] = T(fixed[v]);
            continue;
        }
        int src;
        if (bc == BC_TRANSMISSIVE) src = side == 0 ? 0 : nd - 1;
        else if (bc == BC_REFLECT) src = side == 0 ? gl - 1 : nd - gl;
        else src = side == 0 ? nd - gl : gl - 1;
        const long long gsrc = base + (long long)src * sd;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            T val = U[gsrc + v * a.sv];
            if (bc == BC_REFLECT && v == 1 + d) val = -val;
            U[gdst + v * a.sv] = val;
        }
    }
}

// ------------------------------------------------------- CFL reduction
struct CflArgs {
    const void* U;
    int n[3];
    long long sy, sz, sv, off0;
    double inv_dx[3];
    double gamma;
    DevTime* tm;
};

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = maxT(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_cfl(CflArgs a)
{
    constexpr int NV = DIM + 2;
    if (a.tm->status != 0) return;
    const T* U = reinterpret_cast<const T*>(a.U);
    const long long nx = a.n[0], ny = a.n[1];
    const long long total = nx * ny * (long long)a.n[2];
    const T gamma = T(a.gamma), gm1 = gamma - T(1);
    T idx_[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) idx_[k] = T(a.inv_dx[k]);
    double smax = 0.0;
    bool bad = false;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
        const long long i = id % nx, j = (id / nx) % ny, k = id / (nx * ny);
        const long long g = a.off0 + i + j * a.sy + k * a.sz;
        T u[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = U[g + v * a.sv];
        const T irho = Ar<T>::rcp(u[0]);
        T ke2 = T(0);
        T vel[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) { vel[d] = u[1 + d] * irho; ke2 = fmaT(u[1 + d], vel[d], ke2); }
        const T p = gm1 * fmaT(T(-0.5), ke2, u[DIM + 1]);
        const T c = Ar<T>::sqrt_(gamma * p * irho);
        T s = T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) s = fmaT(absT(vel[d]) + c, idx_[d], s);
        if (!(u[0] > T(0)) || !(p > T(0)) || !isfinite(s)) bad = true;
        else smax = maxT(smax, (double)s);
    }
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

// dt = CFL / smax clipped to t_end; resets the reduction cell
static __global__ void k_dt(DevTime* tm, double cfl)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double dt = 0.0;
    int clipped = 0;
    if (tm->status == 0 && tm->t < tm->t_end) {
        const double smax = __longlong_as_double((long long)tm->smax_bits);
        if (smax > 0.0) dt = cfl / smax;
        if (tm->t + dt >= tm->t_end) { dt = tm->t_end - tm->t; clipped = 1; }
        if (!(dt > 0.0)) { dt = 0.0; clipped = 0; }
    }
    tm->dt = dt;
    tm->clipped = clipped;
    tm->smax_bits = 0ull;
}

// target time for the steps that follow on the stream
static __global__ void k_set_tend(DevTime* tm, double t_end)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) tm->t_end = t_end;
}

static __global__ void k_post(DevTime* tm)
{
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
template <typename T>
__global__ void k_pack(const T* src, T* dst, int nv, int nx, int ny, int nz, long long sy, long long sz,
                       long long sv, long long off0, int to_ghosted)
{
    const long long cells = (long long)nx * ny * nz;
    const long long total = cells * nv;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
        const long long v = id / cells, c = id % cells;
        const long long i = c % nx, j = (c / nx) % ny, k = c / ((long long)nx * ny);
        const long long g = off0 + i + j * sy + k * sz + v * sv;
        if (to_ghosted) dst[g] = src[id];
        else dst[id] = src[g];
    }
}

}  // namespace wis
