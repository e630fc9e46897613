// icarus_internal.cuh -- device-side data layout and physics of libicarus (sm_103a).
//
// Layout in HBM: every cell field is a structure-of-arrays plane over the padded grid
// (n1+4) x (n2+4) x (n3+4) (two ghost layers per side), index 1 (r) fastest, field-major:
// U[f * nt + ((k + 2) * p2 + (j + 2)) * p1 + (i + 2)]. Face fluxes live in three arrays
// F1[8][n3][n2][n1+1], F2[8][n3][n2+1][n1], F3[8][n3+1][n2][n1]. Grid metrics are small 1-D
// arrays computed on the host in double (products of per-axis factors for volumes and areas).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define NV 8
#define NG 2
#define IC_NPROBE_REC 13

namespace icarus {

enum { RHO = 0, M1 = 1, M2 = 2, M3 = 3, EN = 4, B1 = 5, B2 = 6, B3 = 7 };

// radial edge i (0..n1) of a grid with a refined band [lo, hi]: in the coordinate u (ln r when lg,
// else r) the cell density is f = band_refine inside the band and 1 outside, and edge i is where
// its integral from the inner edge reaches i / n1 of the total. Host (metric tables) and device
// (the allocation-free time step) evaluate the same expression.
__host__ __device__ inline double band_edge_at(int n1, double x1min, double x1max, double lo, double hi, int band_refine,
                                               bool lg, int i)
{
    if (i == 0) return x1min;
    if (i == n1) return x1max;
    const double f = (double)band_refine;
    const double u0 = lg ? log(x1min) : x1min, ua = lg ? log(lo) : lo, ub = lg ? log(hi) : hi;
    const double u1 = lg ? log(x1max) : x1max;
    const double s = ((u1 - u0) + (f - 1.0) * (ub - ua)) * i / n1;   // density integral up to edge i
    const double s_in = ua - u0, s_out = s_in + f * (ub - ua);       // ... at the band's two ends
    const double x = s <= s_in ? u0 + s : (s <= s_out ? ua + (s - s_in) / f : ub + (s - s_out));
    return lg ? exp(x) : x;
}

// per-axis metric arrays (device pointers) in the arithmetic type R: the double tables are the
// host's FP64 values, the float tables their roundings (so single-precision kernels never convert
// on the FP64 pipe). Index convention: padded index ip = i + NG.
template <typename R> struct MetricsT {
    // r (or x): [p1] unless noted
    const R *x1c;   // centres
    const R *a1;    // lower-face area factor, [p1 + 1] (r^2 | 1)
    const R *iv1;   // 1 / volume factor ((r+^3 - r-^3)/3 | dx)
    const R *q1;    // (r+^2 - r-^2)/2 / v1  (| 1)
    const R *gp1;   // (a1[i+1] - a1[i]) / v1 (geometric pressure term in m_r)
    const R *iw1;   // 1 / radial width
    const R *ih2;   // 1 / r_c (| 1)
    const R *ig1;   // 1 / (x1c[i+1] - x1c[i-1])
    const R *gm_r2; // GM / r_c^2
    // theta (or y): [p2] unless noted
    const R *x2c;
    const R *a2;    // lower-face area factor, [p2 + 1] (sin theta- | 1)
    const R *iv2;   // 1 / (cos theta- - cos theta+ | dy)
    const R *q2;    // dtheta / v2 (| 1)
    const R *gq2;   // (a2[j+1] - a2[j]) / v2 (geometric pressure term in m_theta)
    const R *sn;    // sin theta_c (| 1)
    const R *cs;    // cos theta_c (| 0)
    const R *ct;    // cot theta_c (| 0)
    const R *is3;   // 1 / sin theta_c (| 1)
    const R *ig2;   // 1 / (x2c[j+1] - x2c[j-1])
    // phi (or z): [p3]
    const R *x3c;
    const R *ig3;   // 1 / (x3c[k+1] - x3c[k-1])
    R id2, id3, iv3;  // 1/dtheta, 1/dphi, 1/v3 (1/dphi | 1/dz)
    R d2, d3;
    // CME footprint: unit vector of each boundary column centre, [3][n2][n3]
    const R *colvec;
    // Linde diffusion length^2: 1 / (dr^-2 + (r dtheta)^-2 + (r sin(theta) dphi)^-2), [p2][p1]
    const R *ldx2;
    // per (theta, r) cell, index jp * cf_p1 + ip, [CF_N][p2][p1]: the products of per-axis factors
    // the FP64 update and div B use, formed once on the host in the same order as the device
    // would (so the values are the same to the bit): a1 iv1, a1+ iv1, a2 jv, a2+ jv, kv, q1 gq2,
    // ih2 ig2, ih2 is3, jv, with jv = q1 iv2 and kv = q1 q2 iv3; and (CF_ORS, CF_LD*) the rotating
    // frame's and the Linde term's per-cell factors
    const R *cf;
    int cf_p1;
    long long cf_n;
};
using Metrics = MetricsT<double>;

// physics constants in the arithmetic type R
// CF_ORS: Omega r_c sin(theta_c); CF_LD0..2: the Linde coefficient C_d / sum_d dx_d^-2 times the
// inverse central-difference widths ig1, ih2 ig2, ih2 is3 (the last times ig3 of the plane)
enum { CF_AM = 0, CF_AP, CF_BM, CF_BP, CF_KV, CF_Q1GQ2, CF_IH2IG2, CF_IH2IS3, CF_JV, CF_ORS, CF_LD0, CF_LD1, CF_LD2,
       CF_N };

template <typename R> __host__ __device__ inline R cfv(const MetricsT<R> &m, int q, int ip, int jp)
{
    return m.cf[q * m.cf_n + (long long)jp * m.cf_p1 + ip];
}

template <typename R> struct PhysT {
    R gamma, gm1, igm1, omega, divb_coef, rho_floor, p_floor;   // gm1 = gamma - 1, igm1 = 1 / gm1
};

struct Scalars {               // device-resident step state
    double t, dt, t_stop, cfl;
    unsigned long long smax_bits;   // batched form: this member's CFL maximum (bits of a double >= 0)
    unsigned int done;              // last-block counter of the CFL reduction
    int status;                     // bit 0: non-finite state; bit 1: a floor acted (strict_floors)
    unsigned long long floor_hits;
    long long ring_head;            // probe records written so far
    double dt_step;                 // dt of the step just completed (set when t advances)
    unsigned int smax_seen;         // FP64 second-stage update: largest CFL speed estimate published
                                    // by its blocks so far (float bits; zero between launches)
};

struct Params {
    int n1, n2, n3, p1, p2, p3;
    long long nt;
    int geom, bc[6];
    int limiter, flux, gravity, divb, init_vphi, cme_model;
    double gamma, omega, divb_coef, rho_floor, p_floor;
    double r_in;                    // inner radius (AU; x1min of the grid)
    // GLM div-B control (divb = 2): psi at the step start / after stage 1 (padded, the state's
    // type), the damping constant and the smallest cell width
    const void *psi0, *psi1;
    double glm_alpha, glm_dmin;
    Metrics m;
    MetricsT<float> mf;             // float roundings of m
    PhysT<double> ph;
    PhysT<float> phf;
    // boundary driving (code units)
    int n_maps, n_cme;
    const double *t_maps;   // [n_maps]
    const double *maps;     // [n_maps][5][n2][n3] (v_r, rho, p, B_r, B_phi)
    const double *cme;      // [n_cme][10] (t_on, dur, ax, ay, az, cos_hw, v_r, rho, p, R = r_in sin(hw))
    // probes
    int n_probes, n_knots, ring_cap;
    const double *traj;     // [P][K][4] SI
    double *ring;           // [cap][P][13]
    double t0, omega_si, b0, p0;
    Scalars *sc;
    int strict_floors;      // 1: a floor activation sets status bit 1
    int *hstatus;           // device address of a host-mapped copy of sc->status (written each step)
};

template <typename R> __host__ __device__ inline const MetricsT<R> &met(const Params &P);
template <> __host__ __device__ inline const MetricsT<double> &met<double>(const Params &P) { return P.m; }
template <> __host__ __device__ inline const MetricsT<float> &met<float>(const Params &P) { return P.mf; }
template <typename R> __host__ __device__ inline const PhysT<R> &phys(const Params &P);
template <> __host__ __device__ inline const PhysT<double> &phys<double>(const Params &P) { return P.ph; }
template <> __host__ __device__ inline const PhysT<float> &phys<float>(const Params &P) { return P.phf; }

__host__ __device__ inline long long cidx(const Params &P, int i, int j, int k)
{
    return ((long long)(k + NG) * P.p2 + (j + NG)) * P.p1 + (i + NG);
}

// ---- physics (templated on the arithmetic type R) --------------------------------------------
template <typename R> struct Prim { R v[NV]; };   // rho, v1, v2, v3, p, B1, B2, B3

template <typename R> __device__ __forceinline__ R rabs(R x) { return x < R(0) ? -x : x; }
template <typename R> __device__ __forceinline__ R rmax(R a, R b) { return a > b ? a : b; }
template <typename R> __device__ __forceinline__ R rmin(R a, R b) { return a < b ? a : b; }

// Reciprocal 1/q with four FP64 operations: q = +-m 2^E with m in [1, 2); y ~ 1/m from the
// single-precision rcp.approx on m's leading 23 bits, r = +-y 2^-E assembled on the integer pipe,
// then two Newton steps t = 1 - q r, r += r t (Markstein, IBM J. Res. Dev. 34 (1990)): the
// estimate error e becomes e^2 (~6e-14), then e^4, so only the final rounding remains: within one
// ulp of the correctly rounded reciprocal (equal to it in about 99.3 % of cases). q outside [2^-1021, 2^1021] in magnitude (zero,
// subnormal, huge, non-finite) takes the library division.
__device__ __forceinline__ double rcp_nr(double q)
{
    const int hi = __double2hiint(q);
    const unsigned int lo = (unsigned int)__double2loint(q);
    const unsigned int e = ((unsigned int)hi >> 20) & 0x7ffu;
    if (e - 2u >= 2043u) return 1.0 / q;
    const int mb = (127 << 23) | ((hi & 0xfffff) << 3) | (int)(lo >> 29);
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(__int_as_float(mb)));
    const int yb = __float_as_int(y);
    const int rhi = (hi & (int)0x80000000) | ((((yb >> 23) & 0xff) + 1919 - (int)e) << 20) | ((yb & 0x7fffff) >> 3);
    double r = __hiloint2double(rhi, yb << 29);
    double t = fma(-q, r, 1.0);
    r = fma(r, t, r);
    t = fma(-q, r, 1.0);
    return fma(r, t, r);
}
__device__ __forceinline__ double rcp_r(double q) { return rcp_nr(q); }
__device__ __forceinline__ float rcp_r(float q) { return 1.f / q; }

// Exact scalings by 1/2 and 4, |x|, max(x, 0) and the larger of two non-negative values, in
// double on the integer pipe (exponent field, sign bit, bit-pattern order), since the FP64 pipe is
// the scarce one; in single precision the plain arithmetic. A scaling is exact whenever its result
// is normal; zero, infinities and NaN pass unchanged; below 2^-1021 (and, for 4x, above 2^1021) the
// double is returned unscaled.
__device__ __forceinline__ double half_r(double x)
{
    const int hi = __double2hiint(x);
    const unsigned int e = ((unsigned int)hi >> 20) & 0x7ffu;
    return e - 2u < 2045u ? __hiloint2double(hi - 0x00100000, __double2loint(x)) : x;
}
__device__ __forceinline__ float half_r(float x) { return 0.5f * x; }
__device__ __forceinline__ double quad_r(double x)
{
    const int hi = __double2hiint(x);
    const unsigned int e = ((unsigned int)hi >> 20) & 0x7ffu;
    return e - 1u < 2044u ? __hiloint2double(hi + 0x00200000, __double2loint(x)) : x;
}
__device__ __forceinline__ float quad_r(float x) { return 4.f * x; }
__device__ __forceinline__ double abs_r(double x)
{
    return __hiloint2double(__double2hiint(x) & 0x7fffffff, __double2loint(x));
}
__device__ __forceinline__ float abs_r(float x) { return rabs(x); }
__device__ __forceinline__ double clamp0_r(double x) { return __double2hiint(x) < 0 ? 0.0 : x; }
__device__ __forceinline__ float clamp0_r(float x) { return rmax(x, 0.f); }
__device__ __forceinline__ double max_nonneg_r(double a, double b)   // a, b >= 0
{
    return __double_as_longlong(a) > __double_as_longlong(b) ? a : b;
}
__device__ __forceinline__ float max_nonneg_r(float a, float b) { return rmax(a, b); }

// conserved -> primitive: v = m / rho, p = (gamma - 1)(e - rho v^2 / 2 - B^2 / 2)
template <typename R> __device__ __forceinline__ void cons2prim(const R *u, R *w, R gm1)
{
    R irho = rcp_r(u[RHO]);
    w[0] = u[RHO];
    w[1] = u[M1] * irho;
    w[2] = u[M2] * irho;
    w[3] = u[M3] * irho;
    R ke = half_r(u[M1] * w[1] + u[M2] * w[2] + u[M3] * w[3]);     // exact halvings (integer pipe in FP64)
    R me = half_r(u[B1] * u[B1] + u[B2] * u[B2] + u[B3] * u[B3]);
    w[4] = gm1 * (u[EN] - ke - me);
    w[5] = u[B1];
    w[6] = u[B2];
    w[7] = u[B3];
}

template <typename R> __device__ __forceinline__ void prim2cons(const R *w, R *u, R igm1)
{
    u[RHO] = w[0];
    u[M1] = w[0] * w[1];
    u[M2] = w[0] * w[2];
    u[M3] = w[0] * w[3];
    u[EN] = w[4] * igm1 + half_r(u[M1] * w[1] + u[M2] * w[2] + u[M3] * w[3])
          + half_r(w[5] * w[5] + w[6] * w[6] + w[7] * w[7]);
    u[B1] = w[5];
    u[B2] = w[6];
    u[B3] = w[7];
}

// Square root of x >= 0 with five FP64 operations, for the wave speeds inside the Riemann flux.
// x = m 2^(2k) with m in [1, 4) is split on the integer pipe (exponent halved exactly, so every
// normal double is in range); y ~ 1/sqrt(m) comes from the single-precision rsqrt.approx (relative
// error below 2^-22.9) on m's leading 23 bits, and r = y 2^-k is widened back on the integer pipe.
// Then two Newton corrections of the root with the coupled reciprocal (Markstein, IBM J. Res. Dev.
// 34 (1990)): s = x r, s += (r / 2)(x - s^2), twice. For an estimate error e the first leaves a
// relative error of about 1.5 e^2 (~3e-14), the second e times that (~1e-21), so the result is the
// correctly rounded root but for the final rounding: within one ulp of it, almost always equal.
// Zero, negative, subnormal and non-finite x take the library sqrt.
__device__ __forceinline__ double sqrt_nr(double x)
{
    const int hi = __double2hiint(x);
    const unsigned int lo = (unsigned int)__double2loint(x);
    if ((unsigned int)hi - 0x00100000u >= 0x7fe00000u) return sqrt(x);   // not positive and normal
    const int e = hi >> 20;
    const int k = (e - 1023) >> 1;
    const int mb = ((127 + e - 1023 - 2 * k) << 23) | ((hi & 0xfffff) << 3) | (int)(lo >> 29);
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(__int_as_float(mb)));
    const int yb = __float_as_int(y);
    const int rhi = ((((yb >> 23) & 0xff) - 127 + 1023 - k) << 20) | ((yb & 0x7fffff) >> 3);
    const int rlo = yb << 29;
    const double r = __hiloint2double(rhi, rlo);               // ~ 1 / sqrt(x)
    const double h = __hiloint2double(rhi - (1 << 20), rlo);   // r / 2
    const double s = x * r;
    const double s1 = fma(h, fma(-s, s, x), s);
    return fma(h, fma(-s1, s1, x), s1);
}

template <bool NR> __device__ __forceinline__ double root(double x) { return NR ? sqrt_nr(x) : sqrt(x); }
template <bool NR> __device__ __forceinline__ float root(float x) { return sqrtf(x); }

// fast magnetosonic speed along direction d:
// c_f^2 = ((a^2 + b^2) + sqrt((a^2 + b^2)^2 - 4 a^2 B_d^2 / rho)) / 2, a^2 = gamma p / rho
// (NR: the FP64 roots by sqrt_nr, used inside the Riemann flux; the time step keeps the library root)
template <typename R, bool NR = false> __device__ __forceinline__ R fast_speed(const R *w, R irho, int d, R gamma)
{
    R a2 = gamma * w[4] * irho;
    R bb = w[5] * w[5] + w[6] * w[6] + w[7] * w[7];
    R s = a2 + bb * irho;
    R bn = w[5 + d];
    if constexpr (NR) {
        const R disc = clamp0_r(s * s - quad_r(a2) * (bn * bn * irho));
        return root<NR>(half_r(s + root<NR>(disc)));
    } else {
        R disc = s * s - R(4) * a2 * (bn * bn * irho);
        disc = rmax(disc, R(0));
        return root<NR>(R(0.5) * (s + root<NR>(disc)));
    }
}

// sign and zero tests on the bit patterns (integer pipe; the FP64 pipe is the scarce one)
__device__ __forceinline__ int hi_bits(double x) { return __double2hiint(x); }
__device__ __forceinline__ int hi_bits(float x) { return __float_as_int(x); }
__device__ __forceinline__ bool is_zero(double x) { return ((__double2hiint(x) & 0x7fffffff) | __double2loint(x)) == 0; }
__device__ __forceinline__ bool is_zero(float x) { return (__float_as_int(x) & 0x7fffffff) == 0; }
__device__ __forceinline__ unsigned long long abs_bits(double x) { return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull; }
__device__ __forceinline__ unsigned int abs_bits(float x) { return (unsigned int)__float_as_int(x) & 0x7fffffffu; }
// binary32 <-> binary64 conversions on the integer pipe (on GB300 the FP64 pipe, which executes
// the hardware conversions, runs at 1/64 of the FP32 rate). widen: exact for normal numbers and
// zeros; subnormal inputs (absent under flush-to-zero arithmetic) give a signed zero; inf and NaN
// keep their class.
__device__ __forceinline__ double widen_f2d(float x)
{
    const unsigned b = __float_as_uint(x), sign = b & 0x80000000u, e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);
    unsigned lo = m << 29;
    if (e == 0u) { hi = sign; lo = 0u; }
    if (e == 0xffu) hi = sign | 0x7ff00000u | (m >> 3) | (m ? 0x80000u : 0u);
    return __hiloint2double((int)hi, (int)lo);
}
// narrow: IEEE round-to-nearest-even from the bit pattern (the 29 dropped mantissa bits decide;
// a carry out of the mantissa moves into the exponent and, at the top, to infinity); results
// below the normal range flush to a signed zero, as flush-to-zero arithmetic does
__device__ __forceinline__ float narrow_d2f(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u, ax = hi & 0x7fffffffu;
    const unsigned base = ((ax - 0x38000000u) << 3) | (lo >> 29);
    const unsigned r = lo & 0x1fffffffu;
    const unsigned up = (r > 0x10000000u || (r == 0x10000000u && (base & 1u))) ? 1u : 0u;
    unsigned bits = sign | (base + up);
    if (ax < 0x38100000u) bits = sign;
    if (ax >= 0x47f00000u) bits = sign | 0x7f800000u | ((ax > 0x7ff00000u || (ax == 0x7ff00000u && lo)) ? 0x400000u : 0u);
    return __uint_as_float(bits);
}

// x <= 0 (for non-NaN x)
template <typename R> __device__ __forceinline__ bool not_positive(R x) { return hi_bits(x) < 0 || is_zero(x); }

// limited slope from the backward and forward differences a, b: zero unless a and b have the
// same sign; van Leer 2ab/(a+b), minmod, or monotonised central
template <typename R> __device__ __forceinline__ R limiter(int lim, R a, R b)
{
    const bool same = (hi_bits(a) ^ hi_bits(b)) >= 0;          // equal sign bits
    if (lim == 1) {                                               // van Leer
        const R s = a + b;
        const R r = R(2) * a * b / s;
        return (same && !is_zero(s)) ? r : R(0);
    }
    if (!same || is_zero(a) || is_zero(b)) return R(0);
    if (lim == 0) return abs_bits(a) < abs_bits(b) ? a : b;      // minmod
    R m = rmin(rmin(R(2) * rabs(a), R(2) * rabs(b)), R(0.5) * rabs(a + b));   // MC
    return hi_bits(a) >= 0 ? m : -m;
}

// HLLD (Miyoshi & Kusano 2005): intermediate states separated by the entropy wave S_M and the
// rotational waves S*_L, S*_R inside S_L = min(u_L, u_R) - max(c_fL, c_fR), S_R = max(u_L, u_R) +
// max(c_fL, c_fR); the normal field of the intermediate states is the mean of the two faces'; a
// degenerate star state (rho (S - u)(S - S_M) - B_n^2 vanishing) keeps the outer tangential
// velocity and field. ul, ur, fl, fr: conserved states and physical fluxes of the face states.
template <typename R>
__device__ __forceinline__ void hlld(const R *wl, const R *wr, const R *ul, const R *ur, const R *fl, const R *fr,
                                     R cl, R cr, int d, R *f)
{
    const int t1 = d == 0 ? 1 : (d == 1 ? 2 : 0), t2 = d == 0 ? 2 : (d == 1 ? 0 : 1);
    const R uL = wl[1 + d], uR = wr[1 + d];
    const R cmax = rmax(cl, cr);
    const R SL = rmin(uL, uR) - cmax, SR = rmax(uL, uR) + cmax;
    if (SL > R(0)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) f[v] = fl[v];
        return;
    }
    if (SR < R(0)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) f[v] = fr[v];
        return;
    }
    const R bn = R(0.5) * (wl[5 + d] + wr[5 + d]);
    const R ptL = wl[4] + R(0.5) * (wl[5] * wl[5] + wl[6] * wl[6] + wl[7] * wl[7]);
    const R ptR = wr[4] + R(0.5) * (wr[5] * wr[5] + wr[6] * wr[6] + wr[7] * wr[7]);
    const R aL = (SL - uL) * wl[0], aR = (SR - uR) * wr[0];
    const R SM = (aR * uR - aL * uL - ptR + ptL) / (aR - aL);
    const R pts = (aR * ptL - aL * ptR + aL * aR * (uR - uL)) / (aR - aL);
    R us[2][NV], vt[2][2], bt[2][2], rs[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const R *w = s ? wr : wl, *u = s ? ur : ul;
        const R S = s ? SR : SL, a = s ? aR : aL, un = w[1 + d], pt = s ? ptR : ptL;
        const R rho = a / (S - SM);
        const R den = a * (S - SM) - bn * bn;
        const R scale = a * (S - un) + bn * bn;
        R vy = w[1 + t1], vz = w[1 + t2], by = w[5 + t1], bz = w[5 + t2];
        if (rabs(den) > R(1e-12) * scale) {
            const R cv = bn * (SM - un) / den, cb = (a * (S - un) - bn * bn) / den;
            vy = w[1 + t1] - by * cv; vz = w[1 + t2] - bz * cv;
            by = w[5 + t1] * cb; bz = w[5 + t2] * cb;
        }
        const R vb = w[1] * w[5] + w[2] * w[6] + w[3] * w[7];
        const R vbs = SM * bn + vy * by + vz * bz;
        const R e = ((S - un) * u[EN] - pt * un + pts * SM + bn * (vb - vbs)) / (S - SM);
        rs[s] = rho;
        vt[s][0] = vy; vt[s][1] = vz; bt[s][0] = by; bt[s][1] = bz;
        us[s][RHO] = rho;
        us[s][M1 + d] = rho * SM; us[s][M1 + t1] = rho * vy; us[s][M1 + t2] = rho * vz;
        us[s][EN] = e;
        us[s][B1 + d] = bn; us[s][B1 + t1] = by; us[s][B1 + t2] = bz;
    }
    const R sqL = sqrt(rs[0]), sqR = sqrt(rs[1]);
    const R SsL = SM - rabs(bn) / sqL, SsR = SM + rabs(bn) / sqR;
    if (SsL >= R(0)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) f[v] = fl[v] + SL * (us[0][v] - ul[v]);
        return;
    }
    if (SsR <= R(0)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) f[v] = fr[v] + SR * (us[1][v] - ur[v]);
        return;
    }
    const R sg = bn > R(0) ? R(1) : (bn < R(0) ? R(-1) : R(0)), isum = R(1) / (sqL + sqR);
    R vss[2], bss[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        vss[c] = (sqL * vt[0][c] + sqR * vt[1][c] + (bt[1][c] - bt[0][c]) * sg) * isum;
        bss[c] = (sqL * bt[1][c] + sqR * bt[0][c] + sqL * sqR * (vt[1][c] - vt[0][c]) * sg) * isum;
    }
    const R vbss = SM * bn + vss[0] * bss[0] + vss[1] * bss[1];
    const bool s = SM < R(0);                       // side of the entropy wave (selects, no indexing)
    const R sq = s ? sqR : sqL, Ss = s ? SsR : SsL, S = s ? SR : SL, rS = s ? rs[1] : rs[0];
    const R vbs = SM * bn + (s ? vt[1][0] * bt[1][0] + vt[1][1] * bt[1][1] : vt[0][0] * bt[0][0] + vt[0][1] * bt[0][1]);
    R uss[NV];
    uss[RHO] = rS;
    uss[M1 + d] = rS * SM; uss[M1 + t1] = rS * vss[0]; uss[M1 + t2] = rS * vss[1];
    uss[EN] = (s ? us[1][EN] : us[0][EN]) + (s ? R(1) : R(-1)) * sq * (vbs - vbss) * sg;
    uss[B1 + d] = bn; uss[B1 + t1] = bss[0]; uss[B1 + t2] = bss[1];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const R uo = s ? ur[v] : ul[v], fo = s ? fr[v] : fl[v], u1 = s ? us[1][v] : us[0][v];
        f[v] = fo + S * (u1 - uo) + Ss * (uss[v] - u1);
    }
}

// Riemann flux across a face normal to d from left / right primitive states.
// single-precision TVDLF with the left and right states in the two lanes of packed FP32
// instructions (x = left, y = right): conserved states, fast speeds and physical fluxes of both
// sides from one instruction stream; the combination (F_L + F_R)/2 - c_max (U_R - U_L)/2 per lane
__device__ __forceinline__ float2 f2_(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ void tvdlf_paired(const float *wl, const float *wr, int d, float gamma, float igm1, float *f)
{
    float2 w[NV], u[NV], F[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v] = f2_(wl[v], wr[v]);
    const float2 h = f2_(0.5f, 0.5f), irho = f2_(1.f / wl[0], 1.f / wr[0]);
    u[RHO] = w[0];
    u[M1] = __fmul2_rn(w[0], w[1]);
    u[M2] = __fmul2_rn(w[0], w[2]);
    u[M3] = __fmul2_rn(w[0], w[3]);
    const float2 mv = __ffma2_rn(u[M1], w[1], __ffma2_rn(u[M2], w[2], __fmul2_rn(u[M3], w[3])));
    const float2 bb = __ffma2_rn(w[5], w[5], __ffma2_rn(w[6], w[6], __fmul2_rn(w[7], w[7])));
    u[EN] = __ffma2_rn(w[4], f2_(igm1, igm1), __fmul2_rn(h, __fadd2_rn(mv, bb)));
    u[B1] = w[5];
    u[B2] = w[6];
    u[B3] = w[7];
    // fast speeds: c_f^2 = (s + sqrt(s^2 - 4 a^2 b_n^2)) / 2, s = a^2 + b^2
    const float2 a2 = __fmul2_rn(__fmul2_rn(f2_(gamma, gamma), w[4]), irho);
    const float2 s = __ffma2_rn(bb, irho, a2);
    const float2 bn = w[5 + d], vn = w[1 + d];
    const float2 nq = __fmul2_rn(__fmul2_rn(f2_(-4.f, -4.f), a2), __fmul2_rn(__fmul2_rn(bn, bn), irho));
    const float2 disc = __ffma2_rn(s, s, nq);
    const float2 cf2 = __fmul2_rn(h, __fadd2_rn(s, f2_(sqrtf(fmaxf(disc.x, 0.f)), sqrtf(fmaxf(disc.y, 0.f)))));
    const float cl = sqrtf(cf2.x), cr = sqrtf(cf2.y);
    // physical fluxes
    const float2 nbn = __fmul2_rn(bn, f2_(-1.f, -1.f));
    const float2 bv = __ffma2_rn(w[5], w[1], __ffma2_rn(w[6], w[2], __fmul2_rn(w[7], w[3])));
    const float2 pt = __ffma2_rn(h, bb, w[4]);
    F[RHO] = __fmul2_rn(u[RHO], vn);
    F[M1] = __ffma2_rn(u[M1], vn, __fmul2_rn(w[5], nbn));
    F[M2] = __ffma2_rn(u[M2], vn, __fmul2_rn(w[6], nbn));
    F[M3] = __ffma2_rn(u[M3], vn, __fmul2_rn(w[7], nbn));
    F[M1 + d] = __fadd2_rn(F[M1 + d], pt);
    F[EN] = __ffma2_rn(__fadd2_rn(u[EN], pt), vn, __fmul2_rn(nbn, bv));
    F[B1] = __ffma2_rn(vn, w[5], __fmul2_rn(nbn, w[1]));
    F[B2] = __ffma2_rn(vn, w[6], __fmul2_rn(nbn, w[2]));
    F[B3] = __ffma2_rn(vn, w[7], __fmul2_rn(nbn, w[3]));
    F[B1 + d] = f2_(0.f, 0.f);       // v_n B_n - B_n v_n: exactly zero
    const float hc = 0.5f * fmaxf(fabsf(vn.x) + cl, fabsf(vn.y) + cr);
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = 0.5f * (F[v].x + F[v].y) - hc * (u[v].y - u[v].x);
}

// TVDLF: (F_L + F_R)/2 - c_max (U_R - U_L)/2; HLL with signal speeds from the fast speeds (flux
// chosen at run time); HLLD when HD (a separate instantiation, so that the larger solver does not
// weigh on the registers of the other two)
template <typename R, bool HD = false>
__device__ __forceinline__ void riemann(const R *wl, const R *wr, int d, int flux, R gamma, R igm1, R *f)
{
    if constexpr (sizeof(R) == 4 && !HD) {
        if (flux == 0) {
            tvdlf_paired(wl, wr, d, gamma, igm1, f);
            return;
        }
    }
    R ul[NV], ur[NV];
    prim2cons(wl, ul, igm1);
    prim2cons(wr, ur, igm1);
    // FP64: 1/rho_L and 1/rho_R from one division, 1 / (rho_L rho_R), while the product stays
    // well inside the normal range (biased exponent test on its bit pattern); two divisions
    // otherwise and in single precision (where a division is cheap)
    R irl, irr;
    if constexpr (sizeof(R) == 8) {
        const R q = wl[0] * wr[0];
        const int ex = (hi_bits(q) >> 20) & 0x7ff;
        if (ex > 60 && ex < 1990) {
            const R iq = rcp_nr(q);
            irl = wr[0] * iq;
            irr = wl[0] * iq;
        } else {
            irl = R(1) / wl[0];
            irr = R(1) / wr[0];
        }
    } else {
        irl = R(1) / wl[0];
        irr = R(1) / wr[0];
    }
    R cl = fast_speed<R, true>(wl, irl, d, gamma), cr = fast_speed<R, true>(wr, irr, d, gamma);
    R fl[NV], fr[NV];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const R *w = s ? wr : wl;
        const R *u = s ? ur : ul;
        R *ff = s ? fr : fl;
        R vn = w[1 + d], bn = w[5 + d];
        R bb = w[5] * w[5] + w[6] * w[6] + w[7] * w[7];
        R bv = w[5] * w[1] + w[6] * w[2] + w[7] * w[3];
        R pt = w[4] + R(0.5) * bb;
        ff[RHO] = u[RHO] * vn;
        ff[M1] = u[M1] * vn - w[5] * bn;
        ff[M2] = u[M2] * vn - w[6] * bn;
        ff[M3] = u[M3] * vn - w[7] * bn;
        ff[M1 + d] += pt;
        ff[EN] = (u[EN] + pt) * vn - bn * bv;
        ff[B1] = vn * w[5] - bn * w[1];
        ff[B2] = vn * w[6] - bn * w[2];
        ff[B3] = vn * w[7] - bn * w[3];
        // the normal component v_n B_n - B_n v_n is exactly zero (the two products are equal; with
        // a fused multiply-add it would come out as the product's rounding error instead)
        ff[B1 + d] = R(0);
    }
    if constexpr (HD) {
        (void)flux;
        hlld<R>(wl, wr, ul, ur, fl, fr, cl, cr, d, f);
    } else if (flux == 0) {
        const R hc = half_r(max_nonneg_r(abs_r(wl[1 + d]) + cl, abs_r(wr[1 + d]) + cr));
#pragma unroll
        for (int v = 0; v < NV; ++v) f[v] = half_r(fl[v] + fr[v]) - hc * (ur[v] - ul[v]);
    } else {
        R sl = rmin(wl[1 + d] - cl, wr[1 + d] - cr);
        R sr = rmax(wl[1 + d] + cl, wr[1 + d] + cr);
        if (sl >= R(0)) {
#pragma unroll
            for (int v = 0; v < NV; ++v) f[v] = fl[v];
        } else if (sr <= R(0)) {
#pragma unroll
            for (int v = 0; v < NV; ++v) f[v] = fr[v];
        } else {
            R idn = R(1) / (sr - sl);
#pragma unroll
            for (int v = 0; v < NV; ++v) f[v] = (sr * fl[v] - sl * fr[v] + sl * sr * (ur[v] - ul[v])) * idn;
        }
    }
}

}  // namespace icarus
