// Marching sweep across x (the y and z directions) in float arithmetic.
//
//   k_march   every lane of a warp takes one grid line (32 consecutive x
//             indices, so every global access of the warp is one coalesced
//             row) and marches along its segment of S cells: each step loads
//             one cell, forms its record (flux, speeds, Roe weights) once,
//             keeps the last six records in registers and computes the face
//             whose six-cell stencil just completed.  The stencil never goes
//             through shared memory.  Linear upwind faces (Eq. linearupwind)
//             finish in the march; faces the detector (Eq. eq27-28) sends to
//             the characteristic regularized WENO-IS flux (Sec. 2.4, Eq.
//             eq8-r) are listed per warp and computed after the march in
//             rounds of QW faces, with one lane per (face, stencil cell),
//             (face, field, sign) and (face, variable) as in k_sweep.  The
//             divergence and the output of the segment's cells follow.
//
// Every face flux, flag and output takes exactly the arithmetic of k_sweep
// (same routines, same operand order), so both kernels give the same bits.
#pragma once

#include "weno_kernels.cuh"

namespace wis {

// cells per marching segment in 2D and 3D (the default tile rule of the host
// code counts lanes with them)
constexpr int kMarchSeg2 = 12, kMarchSeg3 = 18;

// Shared memory of one warp: the face fluxes of its 32 segments, its list of
// WENO faces and the buffers of one round of QW WENO faces.
template <typename T, int DIM, int S>
struct MarchSmem {
    static constexpr int NV = DIM + 2;
    static constexpr int NQ = CellLayout<DIM>::NQ;
    static constexpr int NR = FaceRec<T, DIM>::NR;
    static constexpr int NF = S + 1;                  // faces of a segment of S cells
    static constexpr int QW = DIM == 2 ? 8 : (S > 12 ? 4 : 6);   // WENO faces per round
    static constexpr int FB = NV * NF * 32;           // [NV][NF][lane] face fluxes (x60)
    static constexpr int CR = QW * 6 * NQ;            // [QW][6][NQ] stencil cell records
    static constexpr int FRC = NR * QW;               // [NR][QW] WENO face records
    static constexpr int FPM = QW * NV * 2 * 6;       // [QW][NV][2][6] split fluxes f+-
    static constexpr int RES = QW * NV * 2;           // [QW][NV][2] reconstructions
    static constexpr size_t bytes_t = sizeof(T) * (size_t)(FB + CR + FRC + FPM + RES);
    static constexpr size_t bytes_q = sizeof(int) * (size_t)(32 * NF);   // face list (j * 32 + lane)
    static constexpr size_t per_warp = (bytes_t + bytes_q + 15) / 16 * 16;
};

// One warp per 32 lines x one segment of S cells along DIR (1 or 2); WPB
// warps per CTA, at least MINW resident warps per SM.  Grid: (lines /
// (32 WPB), segments, planes).  No block-wide barrier: the warps of a CTA
// are independent.
template <typename T, int DIM, int DIR, int S, int WPB, bool EXACTDET, int MINW>
__global__ void __launch_bounds__(WPB * 32, MINW / WPB) k_march(SweepArgs a)
{
    static_assert(DIR >= 1 && DIR < DIM, "k_march sweeps across x");
    static_assert((S + 6) % 6 == 0, "the register window rotates every six cells");
    using CL = CellLayout<DIM>;
    using FR = FaceRec<T, DIM>;
    using MS = MarchSmem<T, DIM, S>;
    constexpr int NV = DIM + 2;
    constexpr int NQ = CL::NQ;
    constexpr int NF = MS::NF;
    constexpr int QW = MS::QW;
    constexpr unsigned FULL = 0xffffffffu;

    pdl_enter();
    if (a.tm != nullptr) {
        if (a.tm->status != 0 || !(a.tm->dt > 0.0)) return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* fb = reinterpret_cast<T*>(smem_raw + (size_t)warp * MS::per_warp);
    T* cr = fb + MS::FB;
    T* frc = cr + MS::CR;
    T* fpm = frc + MS::FRC;
    T* res = fpm + MS::FPM;
    int* qid = reinterpret_cast<int*>(res + MS::RES);

    const int nline = a.n[0];
    const int i0 = (blockIdx.x * WPB + warp) * 32;
    if (i0 >= nline) return;   // the whole warp is past the last line
    const int nd = a.n[DIR];
    const bool lvalid = i0 + lane < nline;
    const int line = lvalid ? i0 + lane : nline - 1;   // idle lanes repeat the last line
    const int pb = blockIdx.z;                          // z index (y sweeps) or y index (z sweeps)
    const int c0 = blockIdx.y * S;                      // first cell of the segment
    const int ncell = min(S, nd - c0);
    const long long sd = DIR == 1 ? a.sy : a.sz;
    const long long sp = DIR == 2 ? a.sy : a.sz;
    const long long lbase = a.off0 + line + (long long)pb * sp;
    const T gamma = pick<T>(a.gamma, a.gamma_f);
    const T gm1 = gamma - T(1);
    const T* Ug = reinterpret_cast<const T*>(a.U);
    const T slim = pick<T>(a.slim, a.slim_f);

    // local cell k is cell c0 - 3 + k of the line; ghost cells from the
    // boundary conditions (the branch is uniform over the warp)
    auto load_cell = [&](int k, T* U) {
        const int along = c0 - 3 + k;
        if (along >= 0 && along < nd) {
            const T* p = Ug + lbase + (long long)along * sd;
#pragma unroll
            for (int v = 0; v < NV; ++v) U[v] = p[(long long)v * a.sv];
        } else {
            stage_cell<T, DIM, DIR>(a, Ug, lbase, line, along, nd, U);
        }
    };

    // splitting speeds of a face from the records of its six stencil cells
    // (rec(m, k): entry k of cell m), the Roe state r
    auto speeds = [&](auto rec, const Roe<T, DIM>& r, T& am, T& a0, T& ap) {
        if (a.split == SPLIT_LLF) {
            am = rec(0, CL::LM);
            a0 = rec(0, CL::L0);
            ap = rec(0, CL::LP);
#pragma unroll
            for (int m = 1; m < 6; ++m) {
                am = max_nn(am, rec(m, CL::LM));
                a0 = max_nn(a0, rec(m, CL::L0));
                ap = max_nn(ap, rec(m, CL::LP));
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
    };
    // Eq. eq28 without the 1/60, projected: w = L (U_{j-2} - 5U_{j-1} + ... - U_{j+3})
    auto detector = [&](auto rec, const Roe<T, DIM>& r, T* dU, T* w) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int k = CL::U + v;
            const T u0 = rec(0, k), u1 = rec(1, k), u2 = rec(2, k), u3 = rec(3, k), u4 = rec(4, k), u5 = rec(5, k);
            if (EXACTDET) dU[v] = -fifth_difference(u0, u1, u2, u3, u4, u5);
            else dU[v] = fmaT(T(10), u2 - u3, fmaT(T(5), u4 - u1, u0 - u5));
        }
        proj_all<T, DIM, DIR>(r, dU, w);
    };

    // ---- march: one cell in, one face out per step ------------------------
    unsigned wmask = 0u;   // bit j: face j of the segment takes the WENO flux
    unsigned my_weno = 0u;
    const int last = ncell + 5;
    // face j (between local cells j + 2 and j + 3) from the records of its
    // stencil cells j .. j + 5: rec(m, k) is entry k of cell j + m
    auto face_step = [&](int j, auto rec) {
        auto ga = [&](int k) -> T { return rec(2, k); };
        auto gb = [&](int k) -> T { return rec(3, k); };
        const Roe<T, DIM> rs = roe_state<T, DIM>(ga, gb, gm1);
        T dU[NV], w[NV];
        detector(rec, rs, dU, w);
        const T lim = slim * rs.rt;
        int fmask = 0;
#pragma unroll
        for (int s = 0; s < NV; ++s) fmask |= abs_lt(w[s], lim) ? (1 << s) : 0;
        const bool smooth = a.hybrid != 0 && fmask == (1 << NV) - 1;
        if (smooth) {
            T am, a0, ap;
            speeds(rec, rs, am, a0, ap);
            // Eq. linearupwind: [central six-point flux + sum_s R^s alpha^s (60 dv^s)] / 60
            T Fo[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const int k = CL::F + v;
                const T f05 = rec(0, k) + rec(5, k);
                const T f14 = rec(1, k) + rec(4, k);
                const T f23 = rec(2, k) + rec(3, k);
                Fo[v] = fmaT(T(37), f23, fmaT(T(-8), f14, f05));
            }
            ups_dissipation_add<T, DIM, DIR>(rs, dU, w, am, a0, ap, Fo);
#pragma unroll
            for (int v = 0; v < NV; ++v) fb[(v * NF + j) * 32 + lane] = Fo[v];
        } else {
            wmask |= 1u << j;
        }
        // a face is owned by the segment right of it, the line's last face by the last segment
        if (lvalid && (j < ncell || c0 + j == nd)) {
            if (!smooth) ++my_weno;
            if (a.flags != nullptr) {
                const int face = c0 + j;
                long long fidx;
                if (DIR == 1) fidx = ((long long)pb * (nd + 1) + face) * (long long)a.n[0] + line;
                else fidx = ((long long)face * a.n[1] + pb) * (long long)a.n[0] + line;
                a.flags[fidx] = smooth ? 1 : 0;
            }
        }
    };
    // each cell is loaded one step ahead of its use (two steps ahead: 256^3
    // vortex RHS 2% slower)
    T Ucur[NV], Unx[NV];
    load_cell(0, Unx);
    {
        T q[6][NQ];   // records of the last six cells, slot = local index mod 6
#pragma unroll 1
        for (int g0 = 0; g0 <= last; g0 += 6) {
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                const int K = g0 + r;
                if (K > last) break;
#pragma unroll
                for (int v = 0; v < NV; ++v) Ucur[v] = Unx[v];
                if (K < last) load_cell(K + 1, Unx);
                cell_prepare<T, DIM, DIR>(Ucur, gamma, gm1, q[r]);
                if (K >= 5) face_step(K - 5, [&](int m, int k) -> T { return q[(r + 1 + m) % 6][k]; });
            }
        }
    }

    // ---- WENO faces of the warp's segments ---------------------------------
    if (!lvalid) wmask = 0u;
    const int cnt = __popc(wmask);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    if (total > 0) {
        int pos = incl - cnt;
        for (unsigned m = wmask; m != 0u; m &= m - 1u) qid[pos++] = (__ffs(m) - 1) * 32 + lane;
        __syncwarp();
        const T eps = pick<T>(a.eps, a.eps_f);
        const T lam_scale = pick<T>(a.c_lambda * (1.0 / 3600.0), a.lam_scale_f);
        for (int q0 = 0; q0 < total; q0 += QW) {
            const int qc = total - q0 < QW ? total - q0 : QW;
            // records of the six stencil cells of every face of the round
            for (int it = lane; it < qc * 6; it += 32) {
                const int qq = it / 6, m6 = it - qq * 6;
                const int id = qid[q0 + qq];
                const int jf = id >> 5, lf = id & 31;
                const long long lb = a.off0 + (i0 + lf) + (long long)pb * sp;
                T U[NV], rq[NQ];
                stage_cell<T, DIM, DIR>(a, Ug, lb, i0 + lf, c0 - 3 + jf + m6, nd, U);
                cell_prepare<T, DIM, DIR>(U, gamma, gm1, rq);
#pragma unroll
                for (int k = 0; k < NQ; ++k) cr[(qq * 6 + m6) * NQ + k] = rq[k];
            }
            __syncwarp();
            // per (face, cell): Roe state and splitting speeds of the face,
            // projection of U_m and F_m (Eq. eqchara) and the split fluxes
            // (Eq. flxuspliting, f- stored mirrored); the cell-0 lane of
            // each face also stores the face record for the next two steps
            for (int it = lane; it < qc * 6; it += 32) {
                const int qq = it / 6, m6 = it - qq * 6;
                const T* c6 = cr + qq * 6 * NQ;
                auto rec = [&](int m, int k) -> T { return c6[m * NQ + k]; };
                auto ga = [&](int k) -> T { return c6[2 * NQ + k]; };
                auto gb = [&](int k) -> T { return c6[3 * NQ + k]; };
                const Roe<T, DIM> rs = roe_state<T, DIM>(ga, gb, gm1);
                T am, a0, ap;
                speeds(rec, rs, am, a0, ap);
                am = halve(am);
                a0 = halve(a0);
                ap = halve(ap);
                if (m6 == 0) {
                    T dU[NV], w[NV];
                    detector(rec, rs, dU, w);
                    const T lim = slim * rs.rt;
                    int fmask = 0;
#pragma unroll
                    for (int s = 0; s < NV; ++s) fmask |= abs_lt(w[s], lim) ? (1 << s) : 0;
#pragma unroll
                    for (int k = 0; k < DIM; ++k) frc[(FR::U + k) * QW + qq] = rs.u[k];
                    frc[FR::C * QW + qq] = rs.c;
                    frc[FR::H * QW + qq] = rs.H;
                    frc[FR::HQ2 * QW + qq] = rs.hq2;
#pragma unroll
                    for (int s = 0; s < NV; ++s) frc[(FR::W + s) * QW + qq] = w[s];
                    frc[FR::IRT2 * QW + qq] = Ar<T>::rcp_f(rs.rt * rs.rt);
                    frc[FR::MASK * QW + qq] = T(a.hybrid == 2 ? fmask : 0);
                }
                T xu[NV], xf[NV], wv[NV], wg[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    xu[v] = rec(m6, CL::U + v);
                    xf[v] = rec(m6, CL::F + v);
                }
                proj_all<T, DIM, DIR>(rs, xu, wv);
                proj_all<T, DIM, DIR>(rs, xf, wg);
#pragma unroll
                for (int s = 0; s < NV; ++s) {
                    const T al = s == 0 ? am : (s == NV - 1 ? ap : a0);
                    const T h = halve(wg[s]);
                    const T kk = al * wv[s];
                    fpm[((qq * NV + s) * 2 + 0) * 6 + m6] = h + kk;
                    fpm[((qq * NV + s) * 2 + 1) * 6 + (5 - m6)] = h - kk;
                }
            }
            __syncwarp();
            // one reconstruction per (face, field, sign): Eq. eq6, eq11, eq18, eq8-r
            for (int it = lane; it < qc * NV * 2; it += 32) {
                const int qq = it / (2 * NV);
                const int rem = it - qq * (2 * NV);
                const int s = rem >> 1, sg = rem & 1;
                // Eq. eq27, eq29: lambda^s = c (dv^s / rho~)^2 = c w_s^2 / (3600 rho~^2)
                const T ws = frc[(FR::W + s) * QW + qq];
                const T lam = lam_scale * (ws * ws) * frc[FR::IRT2 * QW + qq];
                const int fm_bits = (int)frc[FR::MASK * QW + qq];
                const int wm = (fm_bits >> s) & 1 ? W_LINEAR : a.wmode;
                const T* v = fpm + ((qq * NV + s) * 2 + sg) * 6;
                res[(qq * NV + s) * 2 + sg] = recon<T>(v[0], v[1], v[2], v[3], v[4], lam, eps, wm);
            }
            __syncwarp();
            // Eq. reconstruction1 and the back-projection Eq. reconstruction2
            for (int it = lane; it < qc * NV; it += 32) {
                const int qq = it / NV, v = it - (it / NV) * NV;
                const int id = qid[q0 + qq];
                const int jf = id >> 5, lf = id & 31;
                Roe<T, DIM> r;
#pragma unroll
                for (int k = 0; k < DIM; ++k) r.u[k] = frc[(FR::U + k) * QW + qq];
                r.c = frc[FR::C * QW + qq];
                r.H = frc[FR::H * QW + qq];
                r.hq2 = frc[FR::HQ2 * QW + qq];
                T wch[NV];
#pragma unroll
                for (int s = 0; s < NV; ++s) wch[s] = res[(qq * NV + s) * 2] + res[(qq * NV + s) * 2 + 1];
                fb[(v * NF + jf) * 32 + lf] = T(60) * back_proj_row<T, DIM, DIR>(r, wch, v);
            }
            __syncwarp();
        }
    }
    my_weno = __reduce_add_sync(FULL, my_weno);
    if (lane == 0 && my_weno != 0u && a.weno_count != nullptr)
        atomicAdd(a.weno_count, (unsigned long long)my_weno);

    // ---- flux divergence and output of the segment's cells ------------------
    const T inv_dx = pick<T>(a.inv_dx * (1.0 / 60.0), a.inv_dx_f);
    T* outp = reinterpret_cast<T*>(a.out);
    T* accp = reinterpret_cast<T*>(a.acc);
    const T* Unp = reinterpret_cast<const T*>(a.Un);
    const T rka = pick<T>(a.rk_a, a.rk_a_f), rkb = pick<T>(a.rk_b, a.rk_b_f);
    const T acs = pick<T>(a.acc_scale, a.acc_scale_f);
    const T dt = a.mode == MODE_COMBINE ? T(a.tm->dt) : T(0);
    bool bad = false;
    // cells in batches of CH: the loads of a batch are issued before its
    // arithmetic and stores (one memory latency per batch, not per cell)
    constexpr int CH = 4;
    if (lvalid) {
        for (int cb = 0; cb < ncell; cb += CH) {
            T la[CH][NV], lu[CH][NV], ln[CH][NV];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (cb + c >= ncell) break;
                const long long g = lbase + (long long)(c0 + cb + c) * sd;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    la[c][v] = T(0);
                    lu[c][v] = T(0);
                    ln[c][v] = T(0);
                    if (accp && a.mode != MODE_ACC_SET) la[c][v] = accp[g + v * a.sv];
                    if (a.mode == MODE_COMBINE) {
                        lu[c][v] = Ug[g + v * a.sv];
                        if (rka != T(0)) ln[c][v] = Unp[g + v * a.sv];
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (cb + c >= ncell) break;
                const long long g = lbase + (long long)(c0 + cb + c) * sd;
                const T* fl = fb + (cb + c) * 32 + lane;   // face cb + c (left of the cell)
                const T* fr = fl + 32;                       // face cb + c + 1
                if (a.mode == MODE_ACC_SET) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) accp[g + v * a.sv] = fl[v * NF * 32] - fr[v * NF * 32];
                    continue;
                }
                T rv[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) rv[v] = (fl[v * NF * 32] - fr[v * NF * 32]) * inv_dx;
                if (a.mode == MODE_ACC_ADD) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) accp[g + v * a.sv] = fmaT(la[c][v], acs, rv[v]);
                } else if (a.mode == MODE_RHS) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) outp[g + v * a.sv] = accp ? fmaT(la[c][v], acs, rv[v]) : rv[v];
                } else {
                    T nu[NV];
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        T tot = rv[v];
                        if (accp) tot = fmaT(la[c][v], acs, tot);
                        T val = rkb * fmaT(dt, tot, lu[c][v]);
                        if (rka != T(0)) val = fmaT(rka, ln[c][v], val);
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
        }
    }
    if (bad) atomicOr(&a.tm->status, 1);
}

// Launch of k_march: segments of 12 cells in 2D and 18 in 3D, two warps per
// CTA.  A segment stages S + 6 cells for its S + 1 faces (the first face is
// also the previous segment's last).  In 3D the 18-cell segments (24 records
// for 19 faces) ran the 256^3 vortex y- and z-sweeps in 0.341 ms against
// 0.367 ms with 12 cells, with 4 WENO faces per round so that 6 CTAs (12
// warps) still fit in shared memory; in 2D 12-cell segments keep 16 warps
// per SM.
template <typename T, int DIM, int DIR, bool EXACTDET>
cudaError_t launch_march(const SweepArgs& a, cudaStream_t s)
{
    constexpr int S = DIM == 3 ? kMarchSeg3 : kMarchSeg2, WPB = 2;
    using MS = MarchSmem<T, DIM, S>;
    // 3D: 12 resident warps per SM leave 160 registers a thread and no
    // spills (256^3 vortex RHS 1.68 -> 1.59 ms against 16 warps at 128
    // registers with spills); 2D fits 128 registers
    auto kern = k_march<T, DIM, DIR, S, WPB, EXACTDET, DIM == 3 ? 12 : 16>;
    const size_t smem = MS::per_warp * WPB;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int nd = a.n[DIR];
    const dim3 grid((unsigned)((a.n[0] + 32 * WPB - 1) / (32 * WPB)), (unsigned)((nd + S - 1) / S),
                    (unsigned)(DIR == 1 ? a.n[2] : a.n[1]));
    return launch_pdl(kern, grid, dim3(32 * WPB), smem, s, a);
}

}  // namespace wis
