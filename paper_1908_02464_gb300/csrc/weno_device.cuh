// Device arithmetic of the regularized WENO-IS characteristic flux.
//
// Everything here is a __device__ __forceinline__ routine used by the sweep
// kernels in weno_kernels.cuh.  The order of operations follows the paper
// (Zhu & Hu, arXiv 1908.02464):
//   cell_prims     direction-independent primitives of one cell
//   cell_record    physical flux and |eigenvalues| along the sweep from them
//   cell_prepare   both (Eq. goveq4 and its multi-D form)
//   roe_state      Roe average at x_{j+1/2} (Sec. 2.4 step (1))
//   proj_all       L^s . x for every field s (Sec. 2.4 step (2)-(3),
//                  Eq. eqchara), written from the structure of L instead of a
//                  dense matrix product
//   back_proj      sum_s R^s w^s (Eq. reconstruction2)
//   recon          candidate fluxes Eq. eq6, indicators Eq. eq11, L2 error
//                  terms Eq. eq18 and regularized weights Eq. eq8-r
//
// Eigenvector convention (fields ordered u-c, u, shear..., u+c):
//   R^{u-c} = (1, u - c n, H - u_n c), R^{u} = (1, u, q^2/2),
//   R^{t}   = (0, e_t, u_t),           R^{u+c} = (1, u + c n, H + u_n c),
//   L = R^{-1}.  With b1 = (gamma-1)/c^2 and
//   t1(x) = b1 (q^2/2 x_rho - u . x_m + x_E),  a(x) = (u_n x_rho - x_mn)/c:
//   L^{u-c} x = (t1 + a)/2,  L^{u} x = x_rho - t1,  L^{t} x = x_mt - u_t x_rho,
//   L^{u+c} x = (t1 - a)/2.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace wis {

// ---------------------------------------------------------------- arithmetic
// Explicit overloads keep float arithmetic in float (no silent promotion).
__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double maxT(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float maxT(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double absT(double a) { return fabs(a); }
__device__ __forceinline__ float absT(float a) { return fabsf(a); }

// x / 2 without the FP64 pipe: for a normal result the exponent field is
// lowered by one on the integer pipes, which is exact; zero stays zero,
// infinities and NaN stay as they are; results below the smallest normal
// number (|x| < 2^-1021, never met by the quantities halved here) become a
// zero of x's sign.  On GB300 a DMUL takes a slot of the narrow FP64 pipe
// that bounds the sweeps, the few integer instructions do not.
__device__ __forceinline__ double halve(double x)
{
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const unsigned ex = (unsigned)hi & 0x7ff00000u;
    int h, l = lo;
    if (ex - 0x00200000u <= 0x7fc00000u) h = hi - 0x00100000;      // normal result
    else if (ex == 0x7ff00000u) h = hi;                             // inf, NaN
    else { h = hi & (int)0x80000000u; l = 0; }                      // zero, tiny
    return __hiloint2double(h, l);
}
__device__ __forceinline__ float halve(float x) { return 0.5f * x; }

template <typename T> struct Ar;

// Reciprocal from the hardware's approximate value (rcp.approx) refined by
// one third-order step of the series 1/d = x / (1 - e) = x (1 + e + e^2 +
// ...), e = 1 - d x (Householder's method of order 3): the seed's relative
// error e becomes about e^3, far below double rounding, so the result is
// within one ulp.  Three FMAs.  For the finite, positive, normal arguments
// of the sweeps (sums of square roots of densities, weight denominators).
__device__ __forceinline__ double rcp_newton(double d)
{
    double x;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
    const double e = __fma_rn(-d, x, 1.0);   // 1 - d x
    return __fma_rn(x, __fma_rn(e, e, e), x);
}

// 1/sqrt(x) from the hardware's approximate value (rsqrt.approx) refined by
// one third-order step of the binomial series (1 - e)^(-1/2) = 1 + e/2 +
// 3 e^2 / 8 + ..., e = 1 - x r^2 (Householder's method of order 3): the
// seed's error leaves a term of about (5/16) e^3.  Two products and three
// FMAs.  For finite, positive, normal x; zero, negative and non-finite
// arguments give NaN (the admissibility checks reject those states).
__device__ __forceinline__ double rsqrt_refined(double x)
{
    double r;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    const double e = __fma_rn(-x, __dmul_rn(r, r), 1.0);
    const double q = __fma_rn(e, 0.375, 0.5);
    return __fma_rn(__dmul_rn(r, e), q, r);
}

template <> struct Ar<double> {
    static __device__ __forceinline__ double rcp_f(double x) { return rcp_newton(x); }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double rsqrt_(double x) { return rsqrt_refined(x); }
};

template <> struct Ar<float> {
    static __device__ __forceinline__ float rcp_f(float x) { return __fdividef(1.0f, x); }
    static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
};

// ------------------------------------------------------------- cell records
// Per-cell quantities kept in shared memory for a sweep along direction DIR.
// Record layout (NQ entries): U[NV], F[NV], sqrt(rho) u[DIM], sqrt(rho) H,
// sqrt(rho), |u_n - c|, |u_n|, |u_n + c|.  The sqrt(rho)-weighted velocity
// and enthalpy make the Roe average of a face two sums and one scaling.
template <int DIM> struct CellLayout {
    static constexpr int NV = DIM + 2;
    static constexpr int U = 0;
    static constexpr int F = NV;
    static constexpr int SU = 2 * NV;
    static constexpr int SH = 2 * NV + DIM;
    static constexpr int SQ = SH + 1;
    static constexpr int LM = SH + 2;   // |u_n - c|
    static constexpr int L0 = SH + 3;   // |u_n|
    static constexpr int LP = SH + 4;   // |u_n + c|
    static constexpr int NQ = SH + 5;
};

// Direction-independent primitives of one cell (NP entries): 1/rho, p, c,
// sqrt(rho) u[DIM], sqrt(rho) H, sqrt(rho).  They are the part of a cell
// record that costs square roots and reciprocals.  The grid solver computes
// them once per cell and Runge-Kutta stage, in the epilogue of the sweep
// that writes the stage's state, and every sweep of the next stage reads
// them instead of recomputing them per direction.
template <int DIM> struct PrimLayout {
    static constexpr int IRHO = 0;
    static constexpr int P = 1;
    static constexpr int C = 2;
    static constexpr int SU = 3;            // sqrt(rho) u[DIM]
    static constexpr int SH = 3 + DIM;      // sqrt(rho) H
    static constexpr int SQ = 4 + DIM;      // sqrt(rho)
    static constexpr int NP = 5 + DIM;
    // stored per cell as one record of 8 values (64 bytes in FP64, the 2D
    // record padded): a cell's primitives are two 32-byte sectors, written
    // and read with 16-byte accesses
    static constexpr int STRIDE = 8;
};

// the primitive record of cell g (PrimLayout::STRIDE values from P + STRIDE g)
template <int DIM>
__device__ __forceinline__ void load_prims(const double* P, long long g, double* out)
{
    const double2* p = reinterpret_cast<const double2*>(P + g * PrimLayout<DIM>::STRIDE);
#pragma unroll
    for (int j = 0; j < PrimLayout<DIM>::STRIDE / 2; ++j) {
        const double2 v = __ldg(p + j);
        if (2 * j < PrimLayout<DIM>::NP) out[2 * j] = v.x;
        if (2 * j + 1 < PrimLayout<DIM>::NP) out[2 * j + 1] = v.y;
    }
}
template <int DIM>
__device__ __forceinline__ void load_prims(const float* P, long long g, float* out)
{
    const float4* p = reinterpret_cast<const float4*>(P + g * PrimLayout<DIM>::STRIDE);
#pragma unroll
    for (int j = 0; j < PrimLayout<DIM>::STRIDE / 4; ++j) {
        const float4 v = __ldg(p + j);
        const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (4 * j + k < PrimLayout<DIM>::NP) out[4 * j + k] = w[k];
    }
}
template <int DIM>
__device__ __forceinline__ void store_prims(double* P, long long g, const double* in)
{
    double2* p = reinterpret_cast<double2*>(P + g * PrimLayout<DIM>::STRIDE);
#pragma unroll
    for (int j = 0; j < PrimLayout<DIM>::STRIDE / 2; ++j) {
        const double x = 2 * j < PrimLayout<DIM>::NP ? in[2 * j] : 0.0;
        const double y = 2 * j + 1 < PrimLayout<DIM>::NP ? in[2 * j + 1] : 0.0;
        p[j] = make_double2(x, y);
    }
}
template <int DIM>
__device__ __forceinline__ void store_prims(float* P, long long g, const float* in)
{
    float4* p = reinterpret_cast<float4*>(P + g * PrimLayout<DIM>::STRIDE);
#pragma unroll
    for (int j = 0; j < PrimLayout<DIM>::STRIDE / 4; ++j) {
        float w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = 4 * j + k < PrimLayout<DIM>::NP ? in[4 * j + k] : 0.0f;
        p[j] = make_float4(w[0], w[1], w[2], w[3]);
    }
}

// Products that the compiler must not fuse with a neighbouring sum into a
// multiply-add.  The cell primitives are computed in several kernels (the
// tile staging, the Runge-Kutta epilogue, k_prims) and read back from memory
// in others; with every product rounded on its own and every fused
// multiply-add written out, all of them give the same bits.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// Primitives of one cell (Eq. goveq4; E = p/(gamma-1) + rho |u|^2/2) into
// P[NP], gm1 = gamma - 1; inv (if not null) receives 1/sqrt(rho) and 1/c.
template <typename T, int DIM>
__device__ __forceinline__ void cell_prims(const T* U, T gamma, T gm1, T* P, T* inv = nullptr)
{
    using PL = PrimLayout<DIM>;
    const T rho = U[0];
    const T isq = Ar<T>::rsqrt_(rho);   // 1/sqrt(rho)
    const T irho = mul_rn(isq, isq);
    T m2 = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) m2 = fmaT(U[1 + k], U[1 + k], m2);
    const T E = U[DIM + 1];
    const T p = mul_rn(gm1, fmaT(-halve(irho), m2, E));
    const T c2 = mul_rn(mul_rn(gamma, p), irho);
    const T ic = Ar<T>::rsqrt_(c2);
    const T c = mul_rn(c2, ic);   // sqrt(c2) without the correctly rounded sqrt sequence
    if (inv != nullptr) { inv[0] = isq; inv[1] = ic; }
    P[PL::IRHO] = irho;
    P[PL::P] = p;
    P[PL::C] = c;
#pragma unroll
    for (int k = 0; k < DIM; ++k) P[PL::SU + k] = mul_rn(U[1 + k], isq);
    P[PL::SH] = mul_rn(E + p, isq);
    P[PL::SQ] = mul_rn(rho, isq);
}

// Cell record for a sweep along DIR (physical flux, |eigenvalues|) from the
// state U and its primitives P.
template <typename T, int DIM, int DIR>
__device__ __forceinline__ void cell_record(const T* U, const T* P, T* q)
{
    using CL = CellLayout<DIM>;
    using PL = PrimLayout<DIM>;
    const T p = P[PL::P], c = P[PL::C];
    const T un = mul_rn(U[1 + DIR], P[PL::IRHO]);
    const T Ep = U[DIM + 1] + p;
#pragma unroll
    for (int v = 0; v < CL::NV; ++v) q[CL::U + v] = U[v];
    q[CL::F + 0] = U[1 + DIR];
#pragma unroll
    for (int k = 0; k < DIM; ++k) q[CL::F + 1 + k] = k == DIR ? fmaT(U[1 + k], un, p) : mul_rn(U[1 + k], un);
    q[CL::F + DIM + 1] = mul_rn(Ep, un);
#pragma unroll
    for (int k = 0; k < DIM; ++k) q[CL::SU + k] = P[PL::SU + k];
    q[CL::SH] = P[PL::SH];
    q[CL::SQ] = P[PL::SQ];
    q[CL::LM] = absT(un - c);
    q[CL::L0] = absT(un);
    q[CL::LP] = absT(un + c);
}

// Primitives, physical flux and |eigenvalues| of one cell: the record of
// cell_record from the primitives of cell_prims.  q[k] receives record
// entry k; inv (if not null) receives 1/sqrt(rho) and 1/c.
template <typename T, int DIM, int DIR>
__device__ __forceinline__ void cell_prepare(const T* U, T gamma, T gm1, T* q, T* inv = nullptr)
{
    T P[PrimLayout<DIM>::NP];
    cell_prims<T, DIM>(U, gamma, gm1, P, inv);
    cell_record<T, DIM, DIR>(U, P, q);
}

// ----------------------------------------------------------------- Roe state
template <typename T, int DIM> struct Roe {
    T u[DIM];
    T c, ic;     // sound speed and 1/c
    T H;
    T b1, hq2;   // (gamma-1)/c^2, |u|^2/2
    T rt;        // Roe density sqrt(rho_a rho_b)
};

// Roe average (Sec. 2.4 step (1)) between cells a (j) and b (j+1); get_a(k)
// and get_b(k) read record entry k of the two cells.
template <typename T, int DIM, typename GA, typename GB>
__device__ __forceinline__ Roe<T, DIM> roe_state(GA get_a, GB get_b, T gm1)
{
    using CL = CellLayout<DIM>;
    Roe<T, DIM> r;
    const T sa = get_a(CL::SQ), sb = get_b(CL::SQ);
    const T inv = Ar<T>::rcp_f(sa + sb);
    T q2 = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        r.u[k] = (get_a(CL::SU + k) + get_b(CL::SU + k)) * inv;
        q2 = fmaT(r.u[k], r.u[k], q2);
    }
    r.H = (get_a(CL::SH) + get_b(CL::SH)) * inv;
    r.hq2 = halve(q2);
    const T c2 = gm1 * (r.H - r.hq2);
    r.ic = Ar<T>::rsqrt_(c2);
    r.c = c2 * r.ic;
    r.b1 = gm1 * r.ic * r.ic;
    r.rt = sa * sb;
    return r;
}

// Order-preserving comparisons and maxima of non-negative values through
// their IEEE bit patterns (integer pipe instead of the floating-point pipe).
__device__ __forceinline__ double max_nn(double a, double b)
{
    return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}
__device__ __forceinline__ float max_nn(float a, float b)
{
    return __int_as_float(max(__float_as_int(a), __float_as_int(b)));
}
__device__ __forceinline__ bool lt_nn(double a, double b) { return __double_as_longlong(a) < __double_as_longlong(b); }
__device__ __forceinline__ bool lt_nn(float a, float b) { return __float_as_int(a) < __float_as_int(b); }
// |w| < lim for a non-negative lim, on the bit patterns (integer pipes only)
__device__ __forceinline__ bool abs_lt(double w, double lim)
{
    return (__double_as_longlong(w) & 0x7fffffffffffffffLL) < __double_as_longlong(lim);
}
__device__ __forceinline__ bool abs_lt(float w, float lim) { return (__float_as_int(w) & 0x7fffffff) < __float_as_int(lim); }

// w[s] = L^s . x for all fields.
template <typename T, int DIM, int DIR>
__device__ __forceinline__ void proj_all(const Roe<T, DIM>& r, const T* x, T* w)
{
    T dot = r.u[0] * x[1];
#pragma unroll
    for (int k = 1; k < DIM; ++k) dot = fmaT(r.u[k], x[1 + k], dot);
    const T t1 = r.b1 * (fmaT(r.hq2, x[0], x[DIM + 1]) - dot);
    const T a = fmaT(r.u[DIR], x[0], -x[1 + DIR]) * r.ic;
    w[0] = halve(t1 + a);
    w[1] = x[0] - t1;
    int s = 2;
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
        if (t == DIR) continue;
        w[s] = fmaT(-r.u[t], x[0], x[1 + t]);
        ++s;
    }
    w[DIM + 1] = halve(t1 - a);
}

// out[v] += sum_s R[v][s] w[s]
template <typename T, int DIM, int DIR>
__device__ __forceinline__ void back_proj_add(const Roe<T, DIM>& r, const T* w, T* out)
{
    constexpr int LAST = DIM + 1;
    const T sum = w[0] + w[1] + w[LAST];
    const T dif = w[LAST] - w[0];
    out[0] += sum;
    int s = 2;
    T eshear = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        T m = r.u[k] * sum;
        if (k == DIR) {
            m = fmaT(r.c, dif, m);
        } else {
            m += w[s];
            eshear = fmaT(r.u[k], w[s], eshear);
            ++s;
        }
        out[1 + k] += m;
    }
    T e = fmaT(r.H, w[0] + w[LAST], r.u[DIR] * r.c * dif);
    e = fmaT(r.hq2, w[1], e);
    out[LAST] += e + eshear;
}

// Row v of sum_s R[v][s] w[s] (Eq. reconstruction2), with the same FP64
// operations for every v so that neighbouring lanes holding different rows
// do not diverge: the row's entries are picked by selects (integer pipe)
// and summed over the fields in their order,
//   R[v][u-c] = base - cn, R[v][u] = ent, R[v][t] = sh_t, R[v][u+c] = base + cn,
// with (base, cn, ent, sh_t) = (1, 0, 1, 0) for v = 0 (mass),
// (u_k, c [k = n], u_k, [k = t]) for v = 1 + k (momentum k) and
// (H, u_n c, q^2/2, u_t) for v = NV - 1 (energy).
template <typename T, int DIM, int DIR>
__device__ __forceinline__ T back_proj_row(const Roe<T, DIM>& r, const T* w, int v)
{
    constexpr int LAST = DIM + 1;
    const T unc = r.u[DIR] * r.c;
    T base = T(1), cn = T(0), ent = T(1);
    T sh[DIM > 1 ? DIM - 1 : 1];
#pragma unroll
    for (int t = 0; t < DIM - 1; ++t) sh[t] = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        if (v == 1 + k) {
            base = r.u[k];
            ent = r.u[k];
            cn = k == DIR ? r.c : T(0);
        }
    }
    int s = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        if (k == DIR) continue;
        if (v == 1 + k) sh[s] = T(1);
        if (v == LAST) sh[s] = r.u[k];
        ++s;
    }
    if (v == LAST) {
        base = r.H;
        cn = unc;
        ent = r.hq2;
    }
    T acc = (base - cn) * w[0];
    acc = fmaT(ent, w[1], acc);
#pragma unroll
    for (int t = 0; t < DIM - 1; ++t) acc = fmaT(sh[t], w[2 + t], acc);
    return fmaT(base + cn, w[LAST], acc);
}

// out += sum_s R^s alpha^s w^s with w = L dU and the entropy and shear fields
// sharing one speed a0 (the LLF, global LF and Roe splittings all do): since
// R w = R L dU = dU, the sum is a0 dU + (am - a0) w_0 R^{u-c} + (ap - a0)
// w_last R^{u+c}, which needs only the two acoustic eigenvectors.
template <typename T, int DIM, int DIR>
__device__ __forceinline__ void ups_dissipation_add(const Roe<T, DIM>& r, const T* dU, const T* w, T am, T a0,
                                                    T ap, T* out)
{
    constexpr int LAST = DIM + 1;
    const T k0 = (am - a0) * w[0], k3 = (ap - a0) * w[LAST];
#pragma unroll
    for (int v = 0; v <= LAST; ++v) out[v] = fmaT(a0, dU[v], out[v]);
    // R^{u-+c} = (1, u -+ c n, H -+ u_n c)
    const T s = k0 + k3, dd = k3 - k0;
    out[0] += s;
#pragma unroll
    for (int k = 0; k < DIM; ++k)
        out[1 + k] = k == DIR ? fmaT(r.u[k], s, fmaT(r.c, dd, out[1 + k])) : fmaT(r.u[k], s, out[1 + k]);
    out[LAST] = fmaT(r.H, s, fmaT(r.u[DIR] * r.c, dd, out[LAST]));
}

// --------------------------------------------------- scalar reconstruction
// Weight modes: 0 regularized (Eq. eq8-r, the method), 1 WENO-IS (Eq. eq8),
// 2 WENO-IS of Wang et al. (Eq. eq14-15), 3 optimal linear weights d_k.
enum { W_REG = 0, W_IS = 1, W_WANG = 2, W_LINEAR = 3 };

// f0..f4 = f_{j-2} .. f_{j+2}; lam = c sigma^s (Eq. eq29).  Returns the
// reconstructed value at x_{j+1/2}.  Every weight rule is written as
// alpha_k = d_k (1 + LT_k / D_k):
//   regularized: D_k = lam beta_k + E_k + eps, LT_k = lam tau_5
//   WENO-IS:     D_k = beta_k + eps,            LT_k = tau_5
//   Wang:        D_k = beta_k + eps,            LT_{0,1} = tau_5^2/(beta_01 + eps), LT_{2,3} = tau_5
template <typename T>
__device__ __forceinline__ T recon(T a, T b, T c, T d, T e, T lam, T eps, int wmode = W_REG);

template <>
__device__ __forceinline__ double recon<double>(double a, double b, double c, double d, double e,
                                                double lam, double eps, int wmode)
{
    // Eq. eq6 with the optimal weights of Eq. eq8 folded in: q_k = d_k fhat_k
    const double q0 = 0.2 * (c + d);                                              // 0.4 (c + d) / 2
    const double q1 = fmaT(0.3, c, -0.1 * b);                                     // 0.2 (3c - b) / 2
    const double q2 = fmaT(0.1, c, fmaT(0.25, d, -0.05 * e));                     // 0.3 (2c + 5d - e) / 6
    const double q3 = fmaT(1.0 / 30.0, a, fmaT(-7.0 / 60.0, b, (11.0 / 60.0) * c));  // 0.1 (2a - 7b + 11c) / 6
    if (wmode == W_LINEAR) return (q0 + q1) + (q2 + q3);
    // Eq. eq11 from shared differences: with d0 = d - c, d1 = c - b,
    //   c - 2d + e = (e - d) - d0,        3c - 4d + e = (c - 2d + e) - 2 d0,
    //   a - 2b + c = (a - b) + d1,        a - 4b + 3c = (a - 2b + c) + 2 d1,
    //   b - 2c + d = d0 - d1,  a - 4b + 6c - 4d + e = (a - 2b + c) - 2 (b - 2c + d) + (c - 2d + e),
    //   -a + 2b - 2d + e = (e - d) - (a - b) - (d0 + d1)
    const double d0 = d - c, d1 = c - b;
    const double b0 = d0 * d0;
    const double b1 = d1 * d1;
    const double ed = e - d, ab = a - b;
    // (s / 2)^2 in place of s^2 / 4: the same bits, the halving off the FP64 pipe
    const double t2 = ed - d0, s2 = halve(fmaT(-2.0, d0, t2));
    const double b2 = fmaT(13.0 / 12.0, t2 * t2, s2 * s2);
    const double t3 = ab + d1, s3 = halve(fmaT(2.0, d1, t3));
    const double b3 = fmaT(13.0 / 12.0, t3 * t3, s3 * s3);
    const double te = d0 - d1;
    double t = fmaT(-2.0, te, t3) + t2;
    double s = halve((ed - ab) - (d0 + d1));
    const double tau = fmaT(13.0 / 12.0, t * t, s * s);
    double D0, D1, D2, D3, L01, L23;
    if (wmode == W_REG) {
        // Eq. eq18 (E_2 = E_3 = 0) and Eq. eq8-r
        const double E = (te * te) * (1.0 / 45.0);
        D0 = fmaT(lam, b0, E + eps);
        D1 = fmaT(lam, b1, E + eps);
        D2 = fmaT(lam, b2, eps);
        D3 = fmaT(lam, b3, eps);
        L01 = L23 = lam * tau;
    } else {
        // Eq. eq8, and Eq. eq14-15 for the two-point stencils
        D0 = b0 + eps; D1 = b1 + eps; D2 = b2 + eps; D3 = b3 + eps;
        L23 = tau;
        if (wmode == W_WANG) {
            t = fmaT(-2.0, c, b + d);
            s = b - d;
            const double b01 = fmaT(13.0 / 12.0, t * t, 0.25 * (s * s));
            L01 = tau * (tau / (b01 + eps));
        } else {
            L01 = tau;
        }
    }
    // sum_k alpha_k fhat_k / sum_k alpha_k over the common denominator
    // P = D_0 D_1 D_2 D_3 (one reciprocal): alpha_k P / d_k = (D_k + L) P / D_k
    // = P + L prod_{j != k} D_j, and the d_k sit in q_k and in the denominator
    const double D01 = D0 * D1, D23 = D2 * D3, P = D01 * D23;
    const double w0 = fmaT(L01, D1 * D23, P);
    const double w1 = fmaT(L01, D0 * D23, P);
    const double w2 = fmaT(L23, D01 * D3, P);
    const double w3 = fmaT(L23, D01 * D2, P);
    const double num = fmaT(w0, q0, fmaT(w1, q1, fmaT(w2, q2, w3 * q3)));
    const double den = fmaT(0.4, w0, fmaT(0.2, w1, fmaT(0.3, w2, 0.1 * w3)));
    return num * rcp_newton(den);
}

template <>
__device__ __forceinline__ float recon<float>(float a, float b, float c, float d, float e,
                                              float lam, float eps, int wmode)
{
    const float q0 = 0.5f * (c + d);
    const float q1 = fmaT(1.5f, c, -0.5f * b);
    const float q2 = fmaT(1.0f / 3.0f, c, fmaT(5.0f / 6.0f, d, (-1.0f / 6.0f) * e));
    const float q3 = fmaT(1.0f / 3.0f, a, fmaT(-7.0f / 6.0f, b, (11.0f / 6.0f) * c));
    if (wmode == W_LINEAR) return fmaT(0.4f, q0, fmaT(0.2f, q1, fmaT(0.3f, q2, 0.1f * q3)));
    const float b0 = (d - c) * (d - c);
    const float b1 = (c - b) * (c - b);
    float t = fmaT(-2.0f, d, c) + e;
    float s = fmaT(-4.0f, d, 3.0f * c) + e;
    const float b2 = fmaT(13.0f / 12.0f, t * t, 0.25f * (s * s));
    t = fmaT(-2.0f, b, a) + c;
    s = fmaT(-4.0f, b, a) + 3.0f * c;
    const float b3 = fmaT(13.0f / 12.0f, t * t, 0.25f * (s * s));
    t = fmaT(-4.0f, b + d, a + e) + 6.0f * c;
    s = fmaT(2.0f, b - d, e - a);
    const float tau = fmaT(13.0f / 12.0f, t * t, 0.25f * (s * s));
    // In float the product of four denominators can underflow (eps = 1e-20),
    // so each ratio LT_k / D_k takes its own reciprocal.
    float D0, D1, D2, D3, L01, L23;
    if (wmode == W_REG) {
        t = fmaT(-2.0f, c, b + d);
        const float E = (t * t) * (1.0f / 45.0f);
        D0 = fmaT(lam, b0, E + eps);
        D1 = fmaT(lam, b1, E + eps);
        D2 = fmaT(lam, b2, eps);
        D3 = fmaT(lam, b3, eps);
        L01 = L23 = lam * tau;
    } else {
        D0 = b0 + eps; D1 = b1 + eps; D2 = b2 + eps; D3 = b3 + eps;
        L23 = tau;
        if (wmode == W_WANG) {
            t = fmaT(-2.0f, c, b + d);
            s = b - d;
            const float b01 = fmaT(13.0f / 12.0f, t * t, 0.25f * (s * s));
            L01 = tau * __fdividef(tau, b01 + eps);
        } else {
            L01 = tau;
        }
    }
    const float a0 = 0.4f * fmaT(L01, __fdividef(1.0f, D0), 1.0f);
    const float a1 = 0.2f * fmaT(L01, __fdividef(1.0f, D1), 1.0f);
    const float a2 = 0.3f * fmaT(L23, __fdividef(1.0f, D2), 1.0f);
    const float a3 = 0.1f * fmaT(L23, __fdividef(1.0f, D3), 1.0f);
    const float num = fmaT(a0, q0, fmaT(a1, q1, fmaT(a2, q2, a3 * q3)));
    const float den = (a0 + a1) + (a2 + a3);
    return num / den;
}

}  // namespace wis
