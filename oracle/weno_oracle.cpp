/*
 * Plain FP64 CPU oracle of the L2-norm regularized WENO-IS Euler solver
 * (Zhu & Hu, "A L2-norm regularized incremental-stencil WENO scheme for
 * compressible flows", arXiv 1908.02464).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the method that the CUDA library is checked against.  Only
 * the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header or constant table with the CUDA
 * library; both are written independently from the paper.
 *
 * Every routine follows the paper's order of operations:
 *   Sec. 2.1  Eq. eq2/eq4   conservative finite-difference semi-discretization
 *   Sec. 2.2  Eq. eq6       incremental-width candidate fluxes
 *             Eq. eq8       WENO-IS weights (comparator, weights=1)
 *             Eq. eq11      closed-form beta_k and tau_5
 *   Sec. 2.3  Eq. eq14-15   Wang et al. modified weights (comparator, weights=2)
 *   Sec. 2.4  steps (1)-(6) Roe average, eigensystem, projection (eqchara),
 *                           flux splitting (flxuspliting), reconstruction
 *                           (reconstruction, reconstruction1) and
 *                           back-projection (reconstruction2)
 *   Sec. 3.1  Eq. eq18      L2-norm error terms, Eq. eq8-r regularized weights
 *   Sec. 3.2  Eq. eq27-29   non-dimensional detector and lambda = c sigma^s
 *   Sec. 3.3  Eq. eqhy, linearupwind, eq31   hybrid switch to the optimal
 *                           linear upwind scheme
 *   Sec. 4    third-order TVD Runge-Kutta, CFL 0.5
 *
 * Readings of points the paper leaves open (the same list is kept with the
 * design notes of the library):
 *   - E_0 = E_1 are evaluated in the squared form (f_{j-1}-2f_j+f_{j+1})^2/45,
 *     which equals the expanded polynomial of Eq. eq18 exactly.
 *   - The second term of Eq. linearupwind carries the factor 1/60 of Eq. eq28
 *     and its lambda^s is the splitting speed alpha^s; with these the linear
 *     scheme is exactly the WENO scheme with omega_k = d_k.
 *   - Per-face hybrid: a face is smooth iff sigma^s < eps_h for every field s.
 *   - LLF speed alpha^s = max over the six stencil cells j-2..j+3 of
 *     |lambda^s(U_m)| (cell eigenvalues u-c, u, u+c).
 *   - Right eigenvectors (1,u-c,H-uc), (1,u,q^2/2), shear (0,e_t,u_t),
 *     (1,u+c,H+uc) with L = R^{-1}; field order u-c, u, shear..., u+c.
 *   - Cell-centred grid x_i = lo + (i+1/2) dx, three ghost layers.
 *   - Shu-Osher TVD RK3, dt = CFL / max sum_d (|u_d|+c)/dx_d from U^n,
 *     clipped to t_end; stage times t, t+dt, t+dt/2.
 *
 * The arithmetic routines are templates over the real type so that the same
 * source, instantiated with an operation-counting type, yields the
 * algorithmic flop counts per cell and per face.
 */
#include <cmath>
#include <cstring>
#include <cstdint>
#include <vector>
#include <algorithm>

/* ------------------------------------------------------------------ */
/* configuration, mirrored by a ctypes structure on the Python side    */
/* ------------------------------------------------------------------ */
extern "C" {
typedef struct {
    int dim;              /* 1, 2, 3 Euler; 0 = scalar linear advection (1D) */
    int n[3];             /* interior cells per direction                    */
    double lo[3], hi[3];  /* domain                                          */
    int bc_lo[3], bc_hi[3];
    double gamma;
    double cfl;
    double eps;           /* epsilon of Eq. eq8 / eq8-r (1e-20)              */
    double c_lambda;      /* c of Eq. eq29 (1)                               */
    double C_thr;         /* C of Eq. eq31 (1)                               */
    double L_char;        /* L of Eq. eq31 (1)                               */
    int alpha_thr;        /* alpha of Eq. eq31 (3)                           */
    int hybrid;           /* 1: switch to the linear scheme on smooth faces;
                             2: per field (linear weights where sigma^s < eps_h) */
    int weights;          /* 0 regularized (eq8-r), 1 WENO-IS (eq8),
                             2 WENO-IS Wang (eq14), 3 linear d_k             */
    int splitting;        /* 0 LLF, 1 global LF, 2 Roe                       */
    double bc_state[2][5];/* conservative inflow states                     */
    double adv_speed;     /* scalar advection speed a, f(u) = a u            */
    double dt_fixed;      /* >0: use this dt instead of the CFL rule         */
} or_cfg;
}

enum { BC_TRANSMISSIVE = 0, BC_REFLECT = 1, BC_PERIODIC = 2, BC_INFLOW = 3,
       BC_DMR_BOTTOM = 4, BC_DMR_TOP = 5, BC_JET = 6 };

/* inflow jet (Mach 2000 jet of Sec. 4.7): bc_state[0] where y < JET_HALF_WIDTH,
 * bc_state[1] elsewhere */
static const double JET_HALF_WIDTH = 0.05;

static const int NG = 3;  /* ghost layers */

/* ------------------------------------------------------------------ */
/* operation-counting real type (for the algorithmic flop counts)      */
/* ------------------------------------------------------------------ */
/* Two tallies per operation kind:
 * - all operations as written (the algorithmic count);
 * - the essential ones: an operation whose operands are both known
 *   constants (built from literals or configuration values) is folded, a
 *   product with a known 0 or +-1, a sum with a known 0 and a quotient by a
 *   known +-1 are structural; neither is counted.  A product with a known 0
 *   is itself a known 0. */
struct OpCount { long long add, mul, div, sqrt_; };
static OpCount g_ops, g_ess;

struct Cnt {
    double v;
    bool k;     /* known constant */
    Cnt() : v(0), k(true) {}
    Cnt(double x) : v(x), k(true) {}
};
static inline Cnt cnt_data(double x) { Cnt c(x); c.k = false; return c; }
static inline bool known(Cnt a, double x) { return a.k && a.v == x; }
static inline Cnt cnt_res(double v, bool k) { Cnt c(v); c.k = k; return c; }
static inline Cnt cnt_add(Cnt a, Cnt b, double r)
{
    g_ops.add++;
    if (!(a.k && b.k) && !known(a, 0.0) && !known(b, 0.0)) g_ess.add++;
    return cnt_res(r, a.k && b.k);
}
static inline Cnt operator+(Cnt a, Cnt b) { return cnt_add(a, b, a.v + b.v); }
static inline Cnt operator-(Cnt a, Cnt b) { return cnt_add(a, b, a.v - b.v); }
static inline Cnt operator*(Cnt a, Cnt b)
{
    g_ops.mul++;
    if (known(a, 0.0) || known(b, 0.0)) return Cnt(0.0);
    if (!(a.k && b.k) && !known(a, 1.0) && !known(a, -1.0) && !known(b, 1.0) && !known(b, -1.0)) g_ess.mul++;
    return cnt_res(a.v * b.v, a.k && b.k);
}
static inline Cnt operator/(Cnt a, Cnt b)
{
    g_ops.div++;
    if (!(a.k && b.k) && !known(b, 1.0) && !known(b, -1.0)) g_ess.div++;
    return cnt_res(a.v / b.v, a.k && b.k);
}
static inline Cnt operator-(Cnt a) { return cnt_res(-a.v, a.k); }
static inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
static inline bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
static inline bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
static inline bool operator<=(Cnt a, Cnt b) { return a.v <= b.v; }
static inline Cnt sqrt_r(Cnt a)
{
    g_ops.sqrt_++;
    if (!a.k) g_ess.sqrt_++;
    return cnt_res(std::sqrt(a.v), a.k);
}
static inline Cnt abs_r(Cnt a) { return cnt_res(std::fabs(a.v), a.k); }
static inline double val(Cnt a) { return a.v; }

/* forward-mode dual number (value, derivative) for Jacobian-vector products;
 * comparisons, max and the hybrid decision act on the value, so flags and
 * LLF maxima are held fixed along the tangent */
struct Dual {
    double v, d;
    Dual() : v(0), d(0) {}
    Dual(double x) : v(x), d(0) {}
    Dual(double x, double dx) : v(x), d(dx) {}
};
static inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
static inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
static inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
static inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
static inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
static inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
static inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
static inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
static inline bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
static inline Dual sqrt_r(Dual a) { double r = std::sqrt(a.v); return Dual(r, 0.5 * a.d / r); }
static inline Dual abs_r(Dual a) { return a.v < 0 ? Dual(-a.v, -a.d) : a; }
static inline double val(Dual a) { return a.v; }

static inline double sqrt_r(double a) { return std::sqrt(a); }
static inline double abs_r(double a) { return std::fabs(a); }
static inline double val(double a) { return a; }

template <class R> static inline R sq(R x) { return x * x; }
template <class R> static inline R maxr(R a, R b) { return (b > a) ? b : a; }

/* ------------------------------------------------------------------ */
/* Sec. 2.2 / 3.1: scalar reconstruction at x_{j+1/2}                  */
/* ------------------------------------------------------------------ */
struct ReconDetail {
    double q[4], beta[4], E[4], tau5, alpha[4], omega[4];
};

/* f[0..4] = f_{j-2}, f_{j-1}, f_j, f_{j+1}, f_{j+2}; lam = regularization
 * parameter of Eq. eq8-r.  Returns the reconstructed flux at x_{j+1/2}. */
template <class R>
static R recon(const R f[5], R lam, int weights, double eps, ReconDetail* det)
{
    const R a = f[0], b = f[1], c = f[2], d = f[3], e = f[4];
    const double dk[4] = {0.4, 0.2, 0.3, 0.1};          /* Eq. eq8 d_k */

    /* Eq. eq6: candidate fluxes of S0..S3 */
    R q[4];
    q[0] = R(0.5) * c + R(0.5) * d;
    q[1] = R(-0.5) * b + R(1.5) * c;
    q[2] = c / R(3.0) + R(5.0) * d / R(6.0) - e / R(6.0);
    q[3] = a / R(3.0) - R(7.0) * b / R(6.0) + R(11.0) * c / R(6.0);

    /* Eq. eq11: smoothness indicators and the global reference tau_5 */
    R beta[4];
    beta[0] = sq(d - c);
    beta[1] = sq(c - b);
    beta[2] = R(13.0) / R(12.0) * sq(c - R(2.0) * d + e)
            + R(0.25) * sq(R(3.0) * c - R(4.0) * d + e);
    beta[3] = R(13.0) / R(12.0) * sq(a - R(2.0) * b + c)
            + R(0.25) * sq(a - R(4.0) * b + R(3.0) * c);
    R tau5 = R(13.0) / R(12.0) * sq(e - R(4.0) * d + R(6.0) * c - R(4.0) * b + a)
           + R(0.25) * sq(e - R(2.0) * d + R(2.0) * b - a);

    /* Eq. eq18: L2-norm error terms (reference stencil S01 for k = 0, 1) */
    R E[4];
    E[0] = sq(b - R(2.0) * c + d) / R(45.0);
    E[1] = E[0];
    E[2] = R(0.0);
    E[3] = R(0.0);

    R alpha[4];
    if (weights == 0) {
        /* Eq. eq8-r */
        for (int k = 0; k < 4; ++k)
            alpha[k] = R(dk[k]) * (R(1.0) + lam * tau5 / (lam * beta[k] + E[k] + R(eps)));
    } else if (weights == 1) {
        /* Eq. eq8 */
        for (int k = 0; k < 4; ++k)
            alpha[k] = R(dk[k]) * (R(1.0) + tau5 / (beta[k] + R(eps)));
    } else if (weights == 2) {
        /* Eq. eq14-15 */
        R beta01 = R(13.0) / R(12.0) * sq(b - R(2.0) * c + d) + R(0.25) * sq(b - d);
        R t01 = tau5 / (beta01 + R(eps));
        alpha[0] = R(dk[0]) * (R(1.0) + tau5 / (beta[0] + R(eps)) * t01);
        alpha[1] = R(dk[1]) * (R(1.0) + tau5 / (beta[1] + R(eps)) * t01);
        alpha[2] = R(dk[2]) * (R(1.0) + tau5 / (beta[2] + R(eps)));
        alpha[3] = R(dk[3]) * (R(1.0) + tau5 / (beta[3] + R(eps)));
    } else {
        /* optimal linear weights */
        for (int k = 0; k < 4; ++k) alpha[k] = R(dk[k]);
    }

    R sum = alpha[0] + alpha[1] + alpha[2] + alpha[3];
    R omega[4];
    for (int k = 0; k < 4; ++k) omega[k] = alpha[k] / sum;

    /* Eq. eq5 */
    R fhat = omega[0] * q[0] + omega[1] * q[1] + omega[2] * q[2] + omega[3] * q[3];

    if (det) {
        for (int k = 0; k < 4; ++k) {
            det->q[k] = val(q[k]); det->beta[k] = val(beta[k]); det->E[k] = val(E[k]);
            det->alpha[k] = val(alpha[k]); det->omega[k] = val(omega[k]);
        }
        det->tau5 = val(tau5);
    }
    return fhat;
}

/* ------------------------------------------------------------------ */
/* governing equations (Eq. goveq4 and its multi-D form)               */
/* ------------------------------------------------------------------ */
static inline int nvar_of(const or_cfg& c) { return c.dim == 0 ? 1 : c.dim + 2; }

template <class R>
struct CellQ {
    R U[5];     /* conservative state                       */
    R F[5];     /* physical flux in the sweep direction     */
    R rho, u[3], p, c, H;
    R lam[5];   /* eigenvalues of the flux Jacobian, field order u-c, u.., u+c */
};

/* primitives, physical flux and eigenvalues of one cell for sweep direction d */
template <class R>
static void cell_quantities(const or_cfg& cf, int d, const R* U, CellQ<R>& q)
{
    const int nv = nvar_of(cf);
    for (int v = 0; v < nv; ++v) q.U[v] = U[v];
    if (cf.dim == 0) {
        q.F[0] = R(cf.adv_speed) * U[0];
        q.lam[0] = R(cf.adv_speed);
        q.rho = R(1.0);
        return;
    }
    const int dim = cf.dim;
    const R gm1 = R(cf.gamma - 1.0);
    q.rho = U[0];
    R q2 = R(0.0);
    for (int k = 0; k < dim; ++k) {
        q.u[k] = U[1 + k] / q.rho;
        q2 += q.u[k] * q.u[k];
    }
    const R E = U[dim + 1];
    q.p = gm1 * (E - R(0.5) * q.rho * q2);
    q.c = sqrt_r(R(cf.gamma) * q.p / q.rho);
    q.H = (E + q.p) / q.rho;
    const R un = q.u[d];
    q.F[0] = U[1 + d];
    for (int k = 0; k < dim; ++k) {
        q.F[1 + k] = U[1 + k] * un;
        if (k == d) q.F[1 + k] = q.F[1 + k] + q.p;
    }
    q.F[dim + 1] = (E + q.p) * un;
    q.lam[0] = un - q.c;
    for (int s = 1; s <= dim; ++s) q.lam[s] = un;
    q.lam[dim + 1] = un + q.c;
}

/* Sec. 2.4 steps (1)-(2): Roe average between cells A (j) and B (j+1) and
 * the left/right eigenvectors of the Roe Jacobian in direction d.
 * Rm[v][s] is component v of right eigenvector s; L[s][v] is component v of
 * left eigenvector s. */
template <class R>
static void roe_eigen(const or_cfg& cf, int d, const CellQ<R>& A, const CellQ<R>& B,
                      R L[5][5], R Rm[5][5], R lam_roe[5], R& rho_t)
{
    const int nv = nvar_of(cf);
    for (int i = 0; i < nv; ++i)
        for (int k = 0; k < nv; ++k) { L[i][k] = R(0.0); Rm[i][k] = R(0.0); }
    if (cf.dim == 0) {
        L[0][0] = R(1.0); Rm[0][0] = R(1.0); lam_roe[0] = R(cf.adv_speed); rho_t = R(1.0);
        return;
    }
    const int dim = cf.dim;
    const R gm1 = R(cf.gamma - 1.0);
    R sa = sqrt_r(A.rho), sb = sqrt_r(B.rho);
    rho_t = sa * sb;
    R u[3];
    R q2 = R(0.0);
    for (int k = 0; k < dim; ++k) {
        u[k] = (sa * A.u[k] + sb * B.u[k]) / (sa + sb);
        q2 += u[k] * u[k];
    }
    R H = (sa * A.H + sb * B.H) / (sa + sb);
    R c2 = gm1 * (H - R(0.5) * q2);
    R c = sqrt_r(c2);
    R un = u[d];
    R b1 = gm1 / c2;
    R b2 = R(0.5) * b1 * q2;
    const int last = dim + 1;

    /* right eigenvectors (columns) */
    Rm[0][0] = R(1.0);
    for (int k = 0; k < dim; ++k) Rm[1 + k][0] = u[k];
    Rm[1 + d][0] = un - c;
    Rm[last][0] = H - un * c;

    Rm[0][1] = R(1.0);
    for (int k = 0; k < dim; ++k) Rm[1 + k][1] = u[k];
    Rm[last][1] = R(0.5) * q2;

    int s = 2;
    for (int t = 0; t < dim; ++t) {
        if (t == d) continue;
        Rm[1 + t][s] = R(1.0);
        Rm[last][s] = u[t];
        ++s;
    }

    Rm[0][last] = R(1.0);
    for (int k = 0; k < dim; ++k) Rm[1 + k][last] = u[k];
    Rm[1 + d][last] = un + c;
    Rm[last][last] = H + un * c;

    /* left eigenvectors (rows), L = R^{-1} */
    L[0][0] = R(0.5) * (b2 + un / c);
    for (int k = 0; k < dim; ++k) L[0][1 + k] = R(-0.5) * (b1 * u[k]);
    L[0][1 + d] = R(-0.5) * (b1 * un + R(1.0) / c);
    L[0][last] = R(0.5) * b1;

    L[1][0] = R(1.0) - b2;
    for (int k = 0; k < dim; ++k) L[1][1 + k] = b1 * u[k];
    L[1][last] = -b1;

    s = 2;
    for (int t = 0; t < dim; ++t) {
        if (t == d) continue;
        L[s][0] = -u[t];
        L[s][1 + t] = R(1.0);
        ++s;
    }

    L[last][0] = R(0.5) * (b2 - un / c);
    for (int k = 0; k < dim; ++k) L[last][1 + k] = R(-0.5) * (b1 * u[k]);
    L[last][1 + d] = R(-0.5) * (b1 * un - R(1.0) / c);
    L[last][last] = R(0.5) * b1;

    lam_roe[0] = un - c;
    for (int k = 1; k <= dim; ++k) lam_roe[k] = un;
    lam_roe[last] = un + c;
}

struct FaceInfo {
    int smooth;           /* 1 = linear upwind scheme used */
    double sigma[5];      /* detector per field, Eq. eq27 */
    double eps_h;
};

/* Numerical flux at x_{j+1/2} in direction d from the six cells
 * S[0..5] = j-2 .. j+3 (Sec. 2.4 steps (1)-(6), Sec. 3.2-3.3). */
template <class R>
static void face_flux(const or_cfg& cf, int d, double eps_h, const CellQ<R>* S,
                      const double* alpha_global, R* Fhat, FaceInfo* info)
{
    const int nv = nvar_of(cf);
    R L[5][5], Rm[5][5], lam_roe[5], rho_t;
    roe_eigen(cf, d, S[2], S[3], L, Rm, lam_roe, rho_t);

    /* Eq. eq28 and eq27: detector.  Fixed evaluation order:
     * dU = (U_{j-2} + 10 U_j + 5 U_{j+2}) - (5 U_{j-1} + 10 U_{j+1} + U_{j+3}) */
    R dU[5], dv[5], sigma[5];
    for (int v = 0; v < nv; ++v) {
        R pos = S[0].U[v] + R(10.0) * S[2].U[v] + R(5.0) * S[4].U[v];
        R neg = R(5.0) * S[1].U[v] + R(10.0) * S[3].U[v] + S[5].U[v];
        dU[v] = pos - neg;
    }
    for (int s = 0; s < nv; ++s) {
        R acc = R(0.0);
        for (int v = 0; v < nv; ++v) acc += L[s][v] * dU[v];
        dv[s] = acc / R(60.0);
        sigma[s] = sq(dv[s] / rho_t);
    }

    /* Eq. flxuspliting: splitting speed per field */
    R alpha[5];
    for (int s = 0; s < nv; ++s) {
        if (cf.splitting == 0) {
            R m = abs_r(S[0].lam[s]);
            for (int k = 1; k < 6; ++k) m = maxr(m, abs_r(S[k].lam[s]));
            alpha[s] = m;
        } else if (cf.splitting == 1) {
            alpha[s] = R(alpha_global[s]);
        } else {
            alpha[s] = abs_r(lam_roe[s]);
        }
    }

    /* Eq. eq31 threshold and the per-face switch of Eq. eqhy */
    int smooth = 0;
    if (cf.hybrid) {
        smooth = 1;
        for (int s = 0; s < nv; ++s)
            if (!(sigma[s] < R(eps_h))) smooth = 0;
    }

    for (int v = 0; v < nv; ++v) Fhat[v] = R(0.0);
    if (smooth) {
        /* Eq. linearupwind (with the 1/60 of Eq. eq28 on the second term) */
        for (int v = 0; v < nv; ++v)
            Fhat[v] = (S[0].F[v] - R(8.0) * S[1].F[v] + R(37.0) * S[2].F[v]
                       + R(37.0) * S[3].F[v] - R(8.0) * S[4].F[v] + S[5].F[v]) / R(60.0);
        for (int s = 0; s < nv; ++s) {
            R w = alpha[s] * dv[s];
            for (int v = 0; v < nv; ++v) Fhat[v] += Rm[v][s] * w;
        }
    } else {
        for (int s = 0; s < nv; ++s) {
            /* Eq. eqchara: project the six cells onto field s */
            R fp[6], fm[6];
            for (int m = 0; m < 6; ++m) {
                R vch = R(0.0), gch = R(0.0);
                for (int v = 0; v < nv; ++v) {
                    vch += L[s][v] * S[m].U[v];
                    gch += L[s][v] * S[m].F[v];
                }
                /* Eq. flxuspliting */
                fp[m] = R(0.5) * (gch + alpha[s] * vch);
                fm[m] = R(0.5) * (gch - alpha[s] * vch);
            }
            /* Eq. eq29 */
            R lam = R(cf.c_lambda) * sigma[s];
            /* per-field hybrid: the linear scheme for a smooth field */
            const int wrule = (cf.hybrid == 2 && sigma[s] < R(eps_h)) ? 3 : cf.weights;
            /* Eq. reconstruction: positive part on j-2..j+2, negative part on
             * the mirrored sequence j+3..j-1 */
            R plus_in[5] = {fp[0], fp[1], fp[2], fp[3], fp[4]};
            R minus_in[5] = {fm[5], fm[4], fm[3], fm[2], fm[1]};
            R fplus = recon(plus_in, lam, wrule, cf.eps, (ReconDetail*)nullptr);
            R fminus = recon(minus_in, lam, wrule, cf.eps, (ReconDetail*)nullptr);
            /* Eq. reconstruction1 */
            R fs = fplus + fminus;
            /* Eq. reconstruction2 */
            for (int v = 0; v < nv; ++v) Fhat[v] += Rm[v][s] * fs;
        }
    }
    if (info) {
        info->smooth = smooth;
        for (int s = 0; s < nv; ++s) info->sigma[s] = val(sigma[s]);
        info->eps_h = eps_h;
    }
}

/* ------------------------------------------------------------------ */
/* grid storage with ghost layers                                      */
/* ------------------------------------------------------------------ */
struct Grid {
    or_cfg c;
    int nv, dim_eff;     /* dim_eff: number of swept directions */
    int n[3], g[3], N[3];
    double dx[3];
    std::vector<double> U;  /* [v][k][j][i] with ghosts */

    explicit Grid(const or_cfg& cf) : c(cf) {
        nv = nvar_of(cf);
        dim_eff = cf.dim == 0 ? 1 : cf.dim;
        for (int a = 0; a < 3; ++a) {
            n[a] = (a < dim_eff) ? cf.n[a] : 1;
            g[a] = (a < dim_eff) ? NG : 0;
            N[a] = n[a] + 2 * g[a];
            dx[a] = (a < dim_eff) ? (cf.hi[a] - cf.lo[a]) / cf.n[a] : 1.0;
        }
        U.assign((size_t)nv * N[0] * N[1] * N[2], 0.0);
    }
    /* i, j, k are interior-based indices (negative for ghosts) */
    size_t idx(int v, int i, int j, int k) const {
        return (((size_t)v * N[2] + (k + g[2])) * N[1] + (j + g[1])) * N[0] + (i + g[0]);
    }
    double& at(int v, int i, int j, int k) { return U[idx(v, i, j, k)]; }
    double at(int v, int i, int j, int k) const { return U[idx(v, i, j, k)]; }
    size_t interior_size() const { return (size_t)n[0] * n[1] * n[2]; }

    void load_interior(const double* Ui) {
        size_t p = 0;
        for (int v = 0; v < nv; ++v)
            for (int k = 0; k < n[2]; ++k)
                for (int j = 0; j < n[1]; ++j)
                    for (int i = 0; i < n[0]; ++i) at(v, i, j, k) = Ui[p++];
    }
    void store_interior(double* Uo) const {
        size_t p = 0;
        for (int v = 0; v < nv; ++v)
            for (int k = 0; k < n[2]; ++k)
                for (int j = 0; j < n[1]; ++j)
                    for (int i = 0; i < n[0]; ++i) Uo[p++] = at(v, i, j, k);
    }
    double center(int a, int i) const { return c.lo[a] + (i + 0.5) * dx[a]; }
};

/* ghost cells of direction a at time t (three layers per side) */
static void fill_ghosts_dir(Grid& G, int a, double t)
{
    const or_cfg& c = G.c;
    const int nv = G.nv;
    const int na = G.n[a];
    int lim[3] = {G.n[0], G.n[1], G.n[2]};
    lim[a] = 1;
    for (int side = 0; side < 2; ++side) {
        const int bc = side == 0 ? c.bc_lo[a] : c.bc_hi[a];
        for (int p2 = 0; p2 < lim[2]; ++p2)
            for (int p1 = 0; p1 < lim[1]; ++p1)
                for (int p0 = 0; p0 < lim[0]; ++p0)
                    for (int gl = 1; gl <= NG; ++gl) {
                        int dst[3] = {p0, p1, p2};
                        int src[3] = {p0, p1, p2};
                        int gi = side == 0 ? -gl : na - 1 + gl;
                        dst[a] = gi;
                        int kind = bc;
                        const double* fixed = nullptr;
                        if (bc == BC_DMR_BOTTOM) {
                            double x = G.center(0, dst[0]);
                            if (x < 1.0 / 6.0) { kind = BC_INFLOW; fixed = c.bc_state[0]; }
                            else kind = BC_REFLECT;
                        } else if (bc == BC_DMR_TOP) {
                            double x = G.center(0, dst[0]);
                            double xs = 1.0 / 6.0 + (1.0 + 20.0 * t) / std::sqrt(3.0);
                            kind = BC_INFLOW;
                            fixed = (x < xs) ? c.bc_state[0] : c.bc_state[1];
                        } else if (bc == BC_INFLOW) {
                            fixed = c.bc_state[0];
                        } else if (bc == BC_JET) {
                            double y = G.dim_eff > 1 ? G.center(1, dst[1]) : 0.0;
                            kind = BC_INFLOW;
                            fixed = (y < JET_HALF_WIDTH) ? c.bc_state[0] : c.bc_state[1];
                        }
                        if (kind == BC_INFLOW) {
                            for (int v = 0; v < nv; ++v)
                                G.at(v, dst[0], dst[1], dst[2]) = fixed[v];
                            continue;
                        }
                        if (kind == BC_TRANSMISSIVE) src[a] = side == 0 ? 0 : na - 1;
                        else if (kind == BC_REFLECT) src[a] = side == 0 ? gl - 1 : na - gl;
                        else src[a] = side == 0 ? na - gl : gl - 1;  /* periodic */
                        for (int v = 0; v < nv; ++v) {
                            double val_ = G.at(v, src[0], src[1], src[2]);
                            if (kind == BC_REFLECT && c.dim > 0 && v == 1 + a) val_ = -val_;
                            G.at(v, dst[0], dst[1], dst[2]) = val_;
                        }
                    }
    }
}

static double eps_h_of(const or_cfg& c, double dx)
{
    /* Eq. eq31 */
    double r = dx / c.L_char;
    double e = c.C_thr;
    for (int k = 0; k < c.alpha_thr; ++k) e *= r;
    return e;
}

/* Eq. goveq5 summed over directions: dU/dt = -sum_d (F_{+1/2} - F_{-1/2}) / dx_d.
 * flags (optional): per direction the faces of shape n with n_d + 1 along d;
 * ratio (optional): max_s sigma^s / eps_h per face. */
static void rhs_grid(Grid& G, double t, std::vector<double>& dU,
                     unsigned char* flags, double* ratio)
{
    const or_cfg& c = G.c;
    const int nv = G.nv;
    for (int a = 0; a < G.dim_eff; ++a) fill_ghosts_dir(G, a, t);
    dU.assign((size_t)nv * G.interior_size(), 0.0);

    size_t face_off = 0;
    for (int a = 0; a < G.dim_eff; ++a) {
        const int na = G.n[a];
        const double eps_h = eps_h_of(c, G.dx[a]);

        /* global LF speeds (Sec. 2.4 step (4), l = whole domain) */
        double alpha_g[5] = {0, 0, 0, 0, 0};
        if (c.splitting == 1) {
            for (int k = 0; k < G.n[2]; ++k)
                for (int j = 0; j < G.n[1]; ++j)
                    for (int i = 0; i < G.n[0]; ++i) {
                        double Uc[5];
                        for (int v = 0; v < nv; ++v) Uc[v] = G.at(v, i, j, k);
                        CellQ<double> q;
                        cell_quantities(c, a, Uc, q);
                        for (int s = 0; s < nv; ++s) alpha_g[s] = std::max(alpha_g[s], std::fabs(q.lam[s]));
                    }
        }

        int lim[3] = {G.n[0], G.n[1], G.n[2]};
        lim[a] = 1;
        int fshape[3] = {G.n[0], G.n[1], G.n[2]};
        fshape[a] = na + 1;
        std::vector<CellQ<double>> line(na + 2 * NG);
        std::vector<double> Fh((size_t)(na + 1) * nv);
        for (int p2 = 0; p2 < lim[2]; ++p2)
            for (int p1 = 0; p1 < lim[1]; ++p1)
                for (int p0 = 0; p0 < lim[0]; ++p0) {
                    /* primitives of every cell of the line, ghosts included */
                    for (int m = -NG; m < na + NG; ++m) {
                        int ix[3] = {p0, p1, p2};
                        ix[a] = m;
                        double Uc[5];
                        for (int v = 0; v < nv; ++v) Uc[v] = G.at(v, ix[0], ix[1], ix[2]);
                        cell_quantities(c, a, Uc, line[m + NG]);
                    }
                    /* face i-1/2 for i = 0..na lies between cells i-1 and i;
                     * its stencil is cells i-3 .. i+2 */
                    for (int i = 0; i <= na; ++i) {
                        FaceInfo info;
                        face_flux(c, a, eps_h, &line[i - 3 + NG], alpha_g, &Fh[(size_t)i * nv], &info);
                        if (flags || ratio) {
                            int fx[3] = {p0, p1, p2};
                            fx[a] = i;
                            size_t fidx = face_off + ((size_t)fx[2] * fshape[1] + fx[1]) * fshape[0] + fx[0];
                            if (flags) flags[fidx] = (unsigned char)info.smooth;
                            if (ratio) {
                                double m = 0.0;
                                for (int s = 0; s < nv; ++s) m = std::max(m, info.sigma[s]);
                                ratio[fidx] = m / eps_h;
                            }
                        }
                    }
                    for (int i = 0; i < na; ++i) {
                        int ix[3] = {p0, p1, p2};
                        ix[a] = i;
                        size_t cell = ((size_t)ix[2] * G.n[1] + ix[1]) * G.n[0] + ix[0];
                        for (int v = 0; v < nv; ++v)
                            dU[(size_t)v * G.interior_size() + cell] -=
                                (Fh[(size_t)(i + 1) * nv + v] - Fh[(size_t)i * nv + v]) / G.dx[a];
                    }
                }
        face_off += (size_t)fshape[0] * fshape[1] * fshape[2];
    }
}

/* Eq. goveq4 state checks: rho > 0, p > 0, all finite */
static int state_ok(const Grid& G)
{
    const or_cfg& c = G.c;
    for (int k = 0; k < G.n[2]; ++k)
        for (int j = 0; j < G.n[1]; ++j)
            for (int i = 0; i < G.n[0]; ++i) {
                double Uc[5];
                for (int v = 0; v < G.nv; ++v) {
                    Uc[v] = G.at(v, i, j, k);
                    if (!std::isfinite(Uc[v])) return 0;
                }
                if (c.dim == 0) continue;
                CellQ<double> q;
                cell_quantities(c, 0, Uc, q);
                if (!(q.rho > 0.0) || !(q.p > 0.0)) return 0;
            }
    return 1;
}

/* wave-speed sum of one conservative state (CFL rule) */
static double state_speed(const Grid& G, const double* Uc)
{
    const or_cfg& c = G.c;
    double s = 0.0;
    for (int a = 0; a < G.dim_eff; ++a) {
        CellQ<double> q;
        cell_quantities(c, a, Uc, q);
        if (c.dim == 0) s += std::fabs(c.adv_speed) / G.dx[a];
        else s += (std::fabs(q.u[a]) + q.c) / G.dx[a];
    }
    return s;
}

/* CFL rule: dt = CFL / max sum_d (|u_d| + c) / dx_d over the interior cells
 * and the fixed boundary states (they enter the domain through the ghost
 * cells; copied ghosts repeat interior speeds) */
static double cfl_dt(const Grid& G)
{
    const or_cfg& c = G.c;
    if (c.dt_fixed > 0.0) return c.dt_fixed;
    double smax = 0.0;
    for (int a = 0; a < G.dim_eff; ++a)
        for (int side = 0; side < 2; ++side) {
            const int bc = side == 0 ? c.bc_lo[a] : c.bc_hi[a];
            const bool s0 = bc == BC_INFLOW || bc == BC_DMR_BOTTOM || bc == BC_DMR_TOP || bc == BC_JET;
            const bool s1 = bc == BC_DMR_TOP || bc == BC_JET;
            if (s0) smax = std::max(smax, state_speed(G, c.bc_state[0]));
            if (s1) smax = std::max(smax, state_speed(G, c.bc_state[1]));
        }
    for (int k = 0; k < G.n[2]; ++k)
        for (int j = 0; j < G.n[1]; ++j)
            for (int i = 0; i < G.n[0]; ++i) {
                double Uc[5];
                for (int v = 0; v < G.nv; ++v) Uc[v] = G.at(v, i, j, k);
                double s = 0.0;
                for (int a = 0; a < G.dim_eff; ++a) {
                    CellQ<double> q;
                    cell_quantities(c, a, Uc, q);
                    if (c.dim == 0) s += std::fabs(c.adv_speed) / G.dx[a];
                    else s += (std::fabs(q.u[a]) + q.c) / G.dx[a];
                }
                smax = std::max(smax, s);
            }
    return c.cfl / smax;
}

/* one third-order TVD Runge-Kutta step (Sec. 4) */
static int rk3_step(Grid& G, double& t, double t_end, double* dt_out)
{
    const int nv = G.nv;
    const size_t ni = G.interior_size();
    double dt = cfl_dt(G);
    /* the step that reaches t_end is clipped and ends exactly at t_end */
    const bool last = (t + dt >= t_end);
    if (last) dt = t_end - t;
    if (!(dt > 0.0)) { if (dt_out) *dt_out = 0.0; return 0; }

    std::vector<double> U0(nv * ni), Ut(nv * ni), L;
    G.store_interior(U0.data());

    rhs_grid(G, t, L, nullptr, nullptr);
    for (size_t p = 0; p < nv * ni; ++p) Ut[p] = U0[p] + dt * L[p];
    G.load_interior(Ut.data());

    rhs_grid(G, t + dt, L, nullptr, nullptr);
    for (size_t p = 0; p < nv * ni; ++p) Ut[p] = 0.75 * U0[p] + 0.25 * (Ut[p] + dt * L[p]);
    G.load_interior(Ut.data());

    rhs_grid(G, t + 0.5 * dt, L, nullptr, nullptr);
    for (size_t p = 0; p < nv * ni; ++p) Ut[p] = U0[p] / 3.0 + 2.0 / 3.0 * (Ut[p] + dt * L[p]);
    G.load_interior(Ut.data());

    if (!state_ok(G)) { G.load_interior(U0.data()); return 3; }
    t = last ? t_end : t + dt;
    if (dt_out) *dt_out = dt;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Jacobian-vector product of the semi-discrete operator: the RHS       */
/* evaluated in dual numbers along the tangent V (ghost cells are       */
/* linear maps of the interior, fixed inflow states carry no tangent).  */
/* ------------------------------------------------------------------ */
static void rhs_jvp_grid(const or_cfg& c, double t, const double* Ui, const double* Vi, double* dU, double* JV)
{
    Grid G(c), H(c);
    G.load_interior(Ui);
    H.load_interior(Vi);
    for (int a = 0; a < G.dim_eff; ++a) {
        fill_ghosts_dir(G, a, t);
        fill_ghosts_dir(H, a, t);
    }
    /* fixed inflow ghosts: zero tangent (the state arrays are otherwise linear) */
    for (int a = 0; a < G.dim_eff; ++a)
        for (int side = 0; side < 2; ++side) {
            const int bc = side == 0 ? c.bc_lo[a] : c.bc_hi[a];
            if (bc != BC_INFLOW && bc != BC_DMR_BOTTOM && bc != BC_DMR_TOP && bc != BC_JET) continue;
            int lim[3] = {G.n[0], G.n[1], G.n[2]};
            lim[a] = 1;
            for (int p2 = 0; p2 < lim[2]; ++p2)
                for (int p1 = 0; p1 < lim[1]; ++p1)
                    for (int p0 = 0; p0 < lim[0]; ++p0)
                        for (int gl = 1; gl <= NG; ++gl) {
                            int ix[3] = {p0, p1, p2};
                            ix[a] = side == 0 ? -gl : G.n[a] - 1 + gl;
                            bool fixed = bc == BC_INFLOW || bc == BC_DMR_TOP || bc == BC_JET;
                            if (bc == BC_DMR_BOTTOM) fixed = G.center(0, ix[0]) < 1.0 / 6.0;
                            if (fixed)
                                for (int v = 0; v < G.nv; ++v) H.at(v, ix[0], ix[1], ix[2]) = 0.0;
                        }
        }
    const int nv = G.nv;
    const size_t ni = G.interior_size();
    for (size_t p = 0; p < nv * ni; ++p) { dU[p] = 0.0; JV[p] = 0.0; }
    for (int a = 0; a < G.dim_eff; ++a) {
        const int na = G.n[a];
        const double eps_h = eps_h_of(c, G.dx[a]);
        int lim[3] = {G.n[0], G.n[1], G.n[2]};
        lim[a] = 1;
        std::vector<CellQ<Dual>> line(na + 2 * NG);
        std::vector<Dual> Fh((size_t)(na + 1) * nv);
        double zeros[5] = {0, 0, 0, 0, 0};
        for (int p2 = 0; p2 < lim[2]; ++p2)
            for (int p1 = 0; p1 < lim[1]; ++p1)
                for (int p0 = 0; p0 < lim[0]; ++p0) {
                    for (int m = -NG; m < na + NG; ++m) {
                        int ix[3] = {p0, p1, p2};
                        ix[a] = m;
                        Dual Uc[5];
                        for (int v = 0; v < nv; ++v)
                            Uc[v] = Dual(G.at(v, ix[0], ix[1], ix[2]), H.at(v, ix[0], ix[1], ix[2]));
                        cell_quantities(c, a, Uc, line[m + NG]);
                    }
                    for (int i = 0; i <= na; ++i)
                        face_flux(c, a, eps_h, &line[i - 3 + NG], zeros, &Fh[(size_t)i * nv], (FaceInfo*)nullptr);
                    for (int i = 0; i < na; ++i) {
                        int ix[3] = {p0, p1, p2};
                        ix[a] = i;
                        size_t cell = ((size_t)ix[2] * G.n[1] + ix[1]) * G.n[0] + ix[0];
                        for (int v = 0; v < nv; ++v) {
                            Dual r = (Fh[(size_t)(i + 1) * nv + v] - Fh[(size_t)i * nv + v]) / Dual(G.dx[a]);
                            dU[(size_t)v * ni + cell] -= r.v;
                            JV[(size_t)v * ni + cell] -= r.d;
                        }
                    }
                }
    }
}

/* ------------------------------------------------------------------ */
/* exact Riemann solver of the 1D Euler equations (Godunov's problem)  */
/* Star pressure from f_L(p) + f_R(p) + u_R - u_L = 0 by Newton's      */
/* method, shock relations (Rankine-Hugoniot) and rarefaction relations*/
/* (isentropic, generalized Riemann invariants).                       */
/* ------------------------------------------------------------------ */
static void pfun(double g, double p, double rk, double pk, double ck, double* f, double* fd)
{
    if (p > pk) {
        double A = 2.0 / ((g + 1.0) * rk);
        double B = (g - 1.0) / (g + 1.0) * pk;
        double s = std::sqrt(A / (p + B));
        *f = (p - pk) * s;
        *fd = s * (1.0 - 0.5 * (p - pk) / (B + p));
    } else {
        double e = (g - 1.0) / (2.0 * g);
        *f = 2.0 * ck / (g - 1.0) * (std::pow(p / pk, e) - 1.0);
        *fd = 1.0 / (rk * ck) * std::pow(p / pk, -(g + 1.0) / (2.0 * g));
    }
}

static int riemann_star(double g, double rl, double ul, double pl, double rr, double ur, double pr,
                        double* ps, double* us)
{
    double cl = std::sqrt(g * pl / rl), cr = std::sqrt(g * pr / rr);
    if (2.0 / (g - 1.0) * (cl + cr) <= ur - ul) return 1;   /* vacuum generated */
    /* two-rarefaction initial guess */
    double e = (g - 1.0) / (2.0 * g);
    double p = std::pow((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) /
                        (cl / std::pow(pl, e) + cr / std::pow(pr, e)), 1.0 / e);
    if (!(p > 0.0)) p = 1e-8 * std::min(pl, pr);
    for (int it = 0; it < 200; ++it) {
        double fl, fdl, fr, fdr;
        pfun(g, p, rl, pl, cl, &fl, &fdl);
        pfun(g, p, rr, pr, cr, &fr, &fdr);
        double pn = p - (fl + fr + ur - ul) / (fdl + fdr);
        if (pn < 0.0) pn = 1e-12 * std::min(pl, pr);
        double ch = 2.0 * std::fabs(pn - p) / (pn + p);
        p = pn;
        if (ch < 1e-15) break;
    }
    double fl, fdl, fr, fdr;
    pfun(g, p, rl, pl, cl, &fl, &fdl);
    pfun(g, p, rr, pr, cr, &fr, &fdr);
    *ps = p;
    *us = 0.5 * (ul + ur) + 0.5 * (fr - fl);
    return 0;
}

static void riemann_sample(double g, double rl, double ul, double pl, double rr, double ur, double pr,
                           double ps, double us, double xi, double* r, double* u, double* p)
{
    double gm = (g - 1.0) / (g + 1.0);
    if (xi <= us) {
        double cl = std::sqrt(g * pl / rl);
        if (ps > pl) {
            double sl = ul - cl * std::sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g));
            if (xi <= sl) { *r = rl; *u = ul; *p = pl; }
            else { *r = rl * (ps / pl + gm) / (gm * ps / pl + 1.0); *u = us; *p = ps; }
        } else {
            double shl = ul - cl;
            double csl = cl * std::pow(ps / pl, (g - 1.0) / (2.0 * g));
            double stl = us - csl;
            if (xi <= shl) { *r = rl; *u = ul; *p = pl; }
            else if (xi > stl) { *r = rl * std::pow(ps / pl, 1.0 / g); *u = us; *p = ps; }
            else {
                double uu = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + xi);
                double cc = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - xi));
                *r = rl * std::pow(cc / cl, 2.0 / (g - 1.0));
                *u = uu;
                *p = pl * std::pow(cc / cl, 2.0 * g / (g - 1.0));
            }
        }
    } else {
        double cr = std::sqrt(g * pr / rr);
        if (ps > pr) {
            double sr = ur + cr * std::sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g));
            if (xi >= sr) { *r = rr; *u = ur; *p = pr; }
            else { *r = rr * (ps / pr + gm) / (gm * ps / pr + 1.0); *u = us; *p = ps; }
        } else {
            double shr = ur + cr;
            double csr = cr * std::pow(ps / pr, (g - 1.0) / (2.0 * g));
            double str = us + csr;
            if (xi >= shr) { *r = rr; *u = ur; *p = pr; }
            else if (xi < str) { *r = rr * std::pow(ps / pr, 1.0 / g); *u = us; *p = ps; }
            else {
                double uu = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + xi);
                double cc = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - xi));
                *r = rr * std::pow(cc / cr, 2.0 / (g - 1.0));
                *u = uu;
                *p = pr * std::pow(cc / cr, 2.0 * g / (g - 1.0));
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* C entry points (ctypes)                                             */
/* ------------------------------------------------------------------ */
extern "C" {

/* reconstruction at x_{j+1/2} from f_{j-2..j+2}; detail[] receives
 * q[4], beta[4], E[4], tau5, alpha[4], omega[4] (21 doubles) */
double or_recon(const double* f, double lam, int weights, double eps, double* detail)
{
    ReconDetail d;
    double r = recon<double>(f, lam, weights, eps, &d);
    if (detail) {
        int p = 0;
        for (int k = 0; k < 4; ++k) detail[p++] = d.q[k];
        for (int k = 0; k < 4; ++k) detail[p++] = d.beta[k];
        for (int k = 0; k < 4; ++k) detail[p++] = d.E[k];
        detail[p++] = d.tau5;
        for (int k = 0; k < 4; ++k) detail[p++] = d.alpha[k];
        for (int k = 0; k < 4; ++k) detail[p++] = d.omega[k];
    }
    return r;
}

/* Roe average eigensystem between conservative states UA, UB (direction d).
 * L, R: nvar*nvar row-major (L[s][v], R[v][s]); lam: nvar; rho_t: 1. */
void or_roe_eigen(const or_cfg* c, int d, const double* UA, const double* UB,
                  double* L, double* R, double* lam, double* rho_t)
{
    CellQ<double> A, B;
    cell_quantities(*c, d, UA, A);
    cell_quantities(*c, d, UB, B);
    double Lm[5][5], Rm[5][5], lr[5], rt;
    roe_eigen(*c, d, A, B, Lm, Rm, lr, rt);
    int nv = nvar_of(*c);
    for (int i = 0; i < nv; ++i) {
        for (int k = 0; k < nv; ++k) { L[i * nv + k] = Lm[i][k]; R[i * nv + k] = Rm[i][k]; }
        lam[i] = lr[i];
    }
    *rho_t = rt;
}

/* physical flux and cell eigenvalues of one conservative state */
void or_cell_flux(const or_cfg* c, int d, const double* U, double* F, double* lam)
{
    CellQ<double> q;
    cell_quantities(*c, d, U, q);
    int nv = nvar_of(*c);
    for (int v = 0; v < nv; ++v) { F[v] = q.F[v]; lam[v] = q.lam[v]; }
}

/* numerical flux of one face from six conservative states U6[m*nvar+v],
 * m = j-2..j+3.  sigma: nvar detector values.  Returns the smooth flag. */
int or_face_flux(const or_cfg* c, int d, double eps_h, const double* U6,
                 const double* alpha_global, double* Fhat, double* sigma)
{
    int nv = nvar_of(*c);
    CellQ<double> S[6];
    for (int m = 0; m < 6; ++m) cell_quantities(*c, d, U6 + m * nv, S[m]);
    FaceInfo info;
    double zeros[5] = {0, 0, 0, 0, 0};
    face_flux(*c, d, eps_h, S, alpha_global ? alpha_global : zeros, Fhat, &info);
    if (sigma) for (int s = 0; s < nv; ++s) sigma[s] = info.sigma[s];
    return info.smooth;
}

double or_eps_h(const or_cfg* c, double dx) { return eps_h_of(*c, dx); }

/* ghost-filled copy of the state: U (interior, [v][k][j][i]) ->
 * Ug ([v][k+gz][j+gy][i+gx] with three ghosts in each swept direction) */
void or_fill_ghosts(const or_cfg* c, double t, const double* U, double* Ug)
{
    Grid G(*c);
    G.load_interior(U);
    for (int a = 0; a < G.dim_eff; ++a) fill_ghosts_dir(G, a, t);
    std::memcpy(Ug, G.U.data(), G.U.size() * sizeof(double));
}

/* semi-discrete right-hand side at time t.  U, dU: interior [v][k][j][i].
 * flags/ratio: optional per-face outputs (see rhs_grid). */
void or_rhs(const or_cfg* c, double t, const double* U, double* dU,
            unsigned char* flags, double* ratio)
{
    Grid G(*c);
    G.load_interior(U);
    std::vector<double> L;
    rhs_grid(G, t, L, flags, ratio);
    std::memcpy(dU, L.data(), L.size() * sizeof(double));
}

/* RHS and its Jacobian-vector product J(U) V at time t (LLF splitting) */
void or_rhs_jvp(const or_cfg* c, double t, const double* U, const double* V, double* dU, double* JV)
{
    rhs_jvp_grid(*c, t, U, V, dU, JV);
}

/* CFL time step of state U (no clipping) */
double or_cfl_dt(const or_cfg* c, const double* U)
{
    Grid G(*c);
    G.load_interior(U);
    return cfl_dt(G);
}

/* one RK3 step in place; returns 0 ok, 3 non-physical (state restored) */
int or_step(const or_cfg* c, double* U, double* t, double t_end, double* dt)
{
    Grid G(*c);
    G.load_interior(U);
    int st = rk3_step(G, *t, t_end, dt);
    G.store_interior(U);
    return st;
}

/* advance to t_end (at most max_steps steps); returns status */
int or_advance(const or_cfg* c, double* U, double* t, double t_end, int max_steps, int* steps)
{
    Grid G(*c);
    G.load_interior(U);
    int k = 0, st = 0;
    while (k < max_steps && *t < t_end) {
        double dt;
        st = rk3_step(G, *t, t_end, &dt);
        if (st) break;
        if (!(dt > 0.0)) break;
        ++k;
    }
    G.store_interior(U);
    if (steps) *steps = k;
    return st;
}

/* conserved totals sum_cells U * dV per variable */
void or_totals(const or_cfg* c, const double* U, double* tot)
{
    Grid G(*c);
    G.load_interior(U);
    double dV = 1.0;
    for (int a = 0; a < G.dim_eff; ++a) dV *= G.dx[a];
    for (int v = 0; v < G.nv; ++v) {
        double s = 0.0;
        for (int k = 0; k < G.n[2]; ++k)
            for (int j = 0; j < G.n[1]; ++j)
                for (int i = 0; i < G.n[0]; ++i) s += G.at(v, i, j, k);
        tot[v] = s * dV;
    }
}

/* algorithmic operation counts: out[0..3] = add/sub, mul, div, sqrt as
 * written; out[4..7] = the essential ones (see Cnt).
 * or_count_cell: per-cell quantities of one cell;
 * or_count_face: one face from six states (cell work excluded); returns the
 * smooth flag so the caller can classify the count (linear or WENO face). */
static void put_counts(long long* out)
{
    out[0] = g_ops.add; out[1] = g_ops.mul; out[2] = g_ops.div; out[3] = g_ops.sqrt_;
    out[4] = g_ess.add; out[5] = g_ess.mul; out[6] = g_ess.div; out[7] = g_ess.sqrt_;
}

void or_count_cell(const or_cfg* c, int d, const double* U, long long* out)
{
    int nv = nvar_of(*c);
    Cnt Uc[5];
    for (int v = 0; v < nv; ++v) Uc[v] = cnt_data(U[v]);
    g_ops = OpCount{0, 0, 0, 0};
    g_ess = OpCount{0, 0, 0, 0};
    CellQ<Cnt> q;
    cell_quantities(*c, d, Uc, q);
    put_counts(out);
}

int or_count_face(const or_cfg* c, int d, double eps_h, const double* U6, long long* out)
{
    int nv = nvar_of(*c);
    CellQ<Cnt> S[6];
    for (int m = 0; m < 6; ++m) {
        Cnt Uc[5];
        for (int v = 0; v < nv; ++v) Uc[v] = cnt_data(U6[m * nv + v]);
        cell_quantities(*c, d, Uc, S[m]);
    }
    double zeros[5] = {0, 0, 0, 0, 0};
    Cnt Fh[5];
    FaceInfo info;
    g_ops = OpCount{0, 0, 0, 0};
    g_ess = OpCount{0, 0, 0, 0};
    face_flux(*c, d, eps_h, S, zeros, Fh, &info);
    put_counts(out);
    return info.smooth;
}

/* exact Riemann problem: star state; returns 1 if the data generate vacuum */
int or_riemann_star(double g, const double* WL, const double* WR, double* ps, double* us)
{
    return riemann_star(g, WL[0], WL[1], WL[2], WR[0], WR[1], WR[2], ps, us);
}

/* exact solution sampled at n points x[] at time t with the interface at x0.
 * W_out: [3][n] primitive (rho, u, p).  Returns 1 on vacuum. */
int or_riemann_sample(double g, const double* WL, const double* WR, double x0, double t,
                      int n, const double* x, double* W_out)
{
    double ps, us;
    if (riemann_star(g, WL[0], WL[1], WL[2], WR[0], WR[1], WR[2], &ps, &us)) return 1;
    for (int i = 0; i < n; ++i) {
        double r, u, p;
        riemann_sample(g, WL[0], WL[1], WL[2], WR[0], WR[1], WR[2], ps, us, (x[i] - x0) / t, &r, &u, &p);
        W_out[i] = r; W_out[n + i] = u; W_out[2 * n + i] = p;
    }
    return 0;
}

} /* extern "C" */
