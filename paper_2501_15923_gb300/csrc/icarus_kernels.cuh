// icarus_kernels.cuh -- the hot-path kernels of libicarus, templated on the state type TS and the
// arithmetic / primitive type TW:
//   FP64  : TS = double, TW = double
//   FP32  : TS = float,  TW = float
//   MIXED : TS = double, TW = float (update accumulation, dt reduction and the primitive recovery
//           of the first four radial cells in double)
// One time step = ghost fill (3 kernels) + face fluxes (3 kernels, one per direction) + div B +
// update, twice (SSP-RK2 stages), then the probe kernel. dt and t stay on the device.
#pragma once
#include <cstdio>

#include "icarus_internal.cuh"
#include "icarus_ops.h"

namespace icarus {

template <typename TS, typename TW> struct Prec {
    static constexpr bool mixed = sizeof(TS) == 8 && sizeof(TW) == 4;
};

// ---------------------------------------------------------------------------------------------
// primitive recovery of one cell in the precision the mode asks for
template <typename TS, typename TW>
__device__ __forceinline__ void recover(const Params &P, const TS *u, TW *w, int i)
{
    if (Prec<TS, TW>::mixed && i < 4) {
        double ud[NV], wd[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) ud[v] = (double)u[v];
        cons2prim<double>(ud, wd, P.ph.gm1);
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = (TW)wd[v];
    } else {
        TW uw[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if constexpr (Prec<TS, TW>::mixed) uw[v] = narrow_d2f(u[v]);
            else uw[v] = (TW)u[v];
        }
        cons2prim<TW>(uw, w, phys<TW>(P).gm1);
    }
}

// ---------------------------------------------------------------------------------------------
// cone CME at the inner boundary column (j, k) at time tau: when the column is inside a CME
// footprint, q (rho, v_r, p, ...) takes the CME values (later CMEs override earlier ones); returns
// whether it is inside any. The footprint: dot product of unit vectors against cos(half-width),
// or (spherical cloud) against the crossing threshold.
__device__ __forceinline__ bool cme_column(const Params &P, double tau, int j, int k, double *q)
{
    const long long per = (long long)P.n2 * P.n3, col = (long long)j * P.n3 + k;
    bool hit = false;
    for (int c = 0; c < P.n_cme; ++c) {
        const double *cm = P.cme + 10 * c;
        if (!(tau >= cm[0] && tau < __dadd_rn(cm[0], cm[1]))) continue;
        double thr = cm[5];
        if (P.cme_model == 1) {
            // spherical cloud: centre at d = r_in - R + v (tau - t_on) on the axis; a column
            // at r_in is inside while cos(alpha) >= (r_in^2 + d^2 - R^2) / (2 r_in d)
            const double r0 = P.r_in, R = cm[9];
            const double d = __dadd_rn(__dsub_rn(r0, R), __dmul_rn(cm[6], __dsub_rn(tau, cm[0])));
            thr = __ddiv_rn(__dsub_rn(__dadd_rn(__dmul_rn(r0, r0), __dmul_rn(d, d)), __dmul_rn(R, R)),
                            __dmul_rn(__dmul_rn(2.0, r0), d));
        }
        double ex = P.m.colvec[col], ey = P.m.colvec[per + col], ez = P.m.colvec[2 * per + col];
        double dot = __dadd_rn(__dadd_rn(__dmul_rn(ex, cm[2]), __dmul_rn(ey, cm[3])), __dmul_rn(ez, cm[4]));
        if (dot >= thr) { q[0] = cm[7]; q[1] = cm[6]; q[2] = cm[8]; hit = true; }
    }
    return hit;
}

// ---------------------------------------------------------------------------------------------
// ghost fill along r: inner side driven by the maps (+ CME) or a plain rule, outer side a plain
// rule. One thread per interior (j, k) column.
template <typename TS, typename TW>
__device__ __forceinline__ void bnd1_col(const Params &P, TS *__restrict__ U, TW *__restrict__ W, int stage, int j, int k,
                                         int task = -1)
{
    const long long nt = P.nt;
    // inner face
    int bc = P.bc[0];
    if (task >= NG) {
        // outer-side layer only
    } else if (bc == 3) {
        double tau = P.sc->t;
        if (stage == 2) tau = __dadd_rn(tau, P.sc->dt);
        // time bracket (clamped outside the table)
        int m0 = 0, m1 = 0;
        double w = 0.0;
        int nm = P.n_maps;
        if (nm > 1 && tau > P.t_maps[0]) {
            if (tau >= P.t_maps[nm - 1]) {
                m0 = m1 = nm - 1;
            } else {
                int m = 0;
                while (m + 1 < nm - 1 && P.t_maps[m + 1] <= tau) ++m;
                m0 = m; m1 = m + 1;
                w = __ddiv_rn(__dsub_rn(tau, P.t_maps[m]), __dsub_rn(P.t_maps[m + 1], P.t_maps[m]));
                w = fmin(fmax(w, 0.0), 1.0);
            }
        }
        const long long per = (long long)P.n2 * P.n3;
        const long long col = (long long)j * P.n3 + k;
        double q[5];
        const int ord[5] = {1, 0, 2, 3, 4};   // maps hold (v_r, rho, p, B_r, B_phi)
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            double a = P.maps[((long long)m0 * 5 + ord[f]) * per + col];
            double b = P.maps[((long long)m1 * 5 + ord[f]) * per + col];
            q[f] = __dadd_rn(__dmul_rn(__dsub_rn(1.0, w), a), __dmul_rn(w, b));
        }
        cme_column(P, tau, j, k, q);
        const double igm1 = 1.0 / (P.gamma - 1.0);
#pragma unroll
        for (int g = 1; g <= NG; ++g) {
            if (task >= 0 && task != g - 1) continue;
            long long cm_ = cidx(P, g - 1, j, k);
            long long cg = cidx(P, -g, j, k);
            double wg[NV], ug[NV];
            wg[0] = q[0]; wg[1] = q[1]; wg[4] = q[2]; wg[5] = q[3]; wg[7] = q[4];
            // asymm: v_theta, v_phi, B_theta of the mirror cell with the sign flipped
            wg[2] = -(double)W[2 * nt + cm_];
            wg[3] = -(double)W[3 * nt + cm_];
            wg[6] = -(double)W[6 * nt + cm_];
            prim2cons<double>(wg, ug, igm1);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                U[v * nt + cg] = (TS)ug[v];
                W[v * nt + cg] = (TW)wg[v];
            }
        }
    } else {
#pragma unroll
        for (int g = 1; g <= NG; ++g) {
            if (task >= 0 && task != g - 1) continue;
            int src = bc == 1 ? 0 : (bc == 2 ? g - 1 : ((-g % P.n1) + P.n1) % P.n1);
            long long cs = cidx(P, src, j, k), cg = cidx(P, -g, j, k);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                TS uu = U[v * nt + cs];
                TW ww = W[v * nt + cs];
                if (bc == 2 && (v == M1 || v == B1)) { uu = -uu; ww = -ww; }
                U[v * nt + cg] = uu;
                W[v * nt + cg] = ww;
            }
        }
    }
    // outer face
    bc = P.bc[1];
#pragma unroll
    for (int g = 1; g <= NG; ++g) {
        if (task >= 0 && task != NG + g - 1) continue;
        int gi = P.n1 - 1 + g;
        int src = bc == 1 ? P.n1 - 1 : (bc == 2 ? P.n1 - g : (gi % P.n1));
        long long cs = cidx(P, src, j, k), cg = cidx(P, gi, j, k);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            TS uu = U[v * nt + cs];
            TW ww = W[v * nt + cs];
            if (bc == 2 && (v == M1 || v == B1)) { uu = -uu; ww = -ww; }
            U[v * nt + cg] = uu;
            W[v * nt + cg] = ww;
        }
        if (bc == 1 && P.geom == 0) {
            // spherical outer radius: B_r continues as r^-2 (r^2 B_r is copied), so the ghost
            // layer adds no divergence; e follows the change of B^2
            const double rs = P.m.x1c[src + NG], rg = P.m.x1c[gi + NG];
            const double f = (rs / rg) * (rs / rg);
            const double bs = (double)U[B1 * nt + cs], bg = bs * f;
            U[EN * nt + cg] = (TS)((double)U[EN * nt + cs] + 0.5 * (bg * bg - bs * bs));
            U[B1 * nt + cg] = (TS)bg;
            W[B1 * nt + cg] = (TW)((double)W[B1 * nt + cs] * f);
        }
    }
}

template <typename TS, typename TW>
__global__ void k_bnd1(Params P, TS *__restrict__ U, TW *__restrict__ W, int stage)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int k = blockIdx.y;
    if (j >= P.n2 || k >= P.n3) return;
    bnd1_col<TS, TW>(P, U, W, stage, j, k, threadIdx.y);     // threadIdx.y: one of the 2 x NG layers
}

// ghost fill along theta (D = 1) or phi (D = 2) by copy / reflection / periodic images.
// D = 1 covers every r (ghosts included) and interior phi; D = 2 covers everything.
template <int D, typename TS, typename TW>
__device__ __forceinline__ void bnd23_cell(const Params &P, TS *__restrict__ U, TW *__restrict__ W, int ip, int o,
                                           int task = -1)
{
    int i = ip - NG;
    const int n = D == 1 ? P.n2 : P.n3;
    const long long nt = P.nt;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        int bc = P.bc[2 * D + side];
#pragma unroll
        for (int g = 1; g <= NG; ++g) {
            if (task >= 0 && task != side * NG + g - 1) continue;
            int gi = side == 0 ? -g : n - 1 + g;
            int src;
            if (bc == 1) src = side == 0 ? 0 : n - 1;
            else if (bc == 2) src = side == 0 ? g - 1 : n - g;
            else src = ((gi % n) + n) % n;
            long long cs, cg;
            if (D == 1) { cs = cidx(P, i, src, o); cg = cidx(P, i, gi, o); }
            else { cs = cidx(P, i, o - NG, src); cg = cidx(P, i, o - NG, gi); }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                TS uu = U[v * nt + cs];
                TW ww = W[v * nt + cs];
                if (bc == 2 && (v == M1 + D || v == B1 + D)) { uu = -uu; ww = -ww; }
                U[v * nt + cg] = uu;
                W[v * nt + cg] = ww;
            }
        }
    }
}

template <int D, typename TS, typename TW>
__global__ void k_bnd23(Params P, TS *__restrict__ U, TW *__restrict__ W)
{
    int ip = blockIdx.x * blockDim.x + threadIdx.x;     // padded r index
    int o = blockIdx.y;                                 // other index
    if (ip >= P.p1) return;
    if (D == 1 && o >= P.n3) return;
    if (D == 2 && o >= P.p2) return;
    bnd23_cell<D, TS, TW>(P, U, W, ip, o, threadIdx.y);       // threadIdx.y: one of the 2 x NG layers
}

// ---------------------------------------------------------------------------------------------
// fused reconstruction + face flux along direction D. Threads sweep S cells along D; each cell's
// limited slopes are computed once, its face states are exchanged through shared memory and
// every thread but the first computes the flux through the lower face of its cell.
// A tile is BX x BY threads; along D it covers S - 1 faces (S = BX for D = 0, BY otherwise).
// D = 0: faces f0 .. f0+BX-2 of BY consecutive (j) rows; D = 1, 2: BY-1 faces along D for BX
// consecutive r. Must be called by every thread of the block (it synchronises the block).
// GLM (template flag, psi of type TP): psi is reconstructed alongside (cell and upper-face values
// of the neighbour in sQW / sQP), and after the Riemann flux the (B_n, psi) star state replaces
// the normal-field flux by psi* and writes c_h^2 B_n* to FP (the GLM div-B control's face step)
template <int D, int BX, int BY, typename TW, bool HD = false, bool GLM = false, typename TP = TW>
__device__ __forceinline__ void flux_tile(const Params &P, const TW *__restrict__ W, TW *__restrict__ F,
                                          int bx, int by, int bz, int tx, int ty, TW *sW, TW *sP,
                                          const TP *__restrict__ Psi = nullptr, TW *__restrict__ FP = nullptr,
                                          TW *sQW = nullptr, TW *sQP = nullptr, TW *sD = nullptr)
{
    constexpr int S = D == 0 ? BX : BY;
    const int ts = D == 0 ? tx : ty;
    int i, j, k, s, nD;
    bool inrange;
    if (D == 0) {
        nD = P.n1;
        s = bx * (S - 1) - 1 + tx;
        i = s; j = by * BY + ty; k = bz;
        inrange = j < P.n2;
    } else if (D == 1) {
        nD = P.n2;
        i = bx * BX + tx;
        s = by * (S - 1) - 1 + ty;
        j = s; k = bz;
        inrange = i < P.n1;
    } else {
        nD = P.n3;
        i = bx * BX + tx;
        s = by * (S - 1) - 1 + ty;
        k = s; j = bz;
        inrange = i < P.n1;
    }
    const bool valid = inrange && s <= nD;
    const long long nt = P.nt;
    const long long st = D == 0 ? 1 : (D == 1 ? (long long)P.p1 : (long long)P.p1 * P.p2);
    const int sl = ty * BX + tx, sz = BX * BY;
    TW wc[NV], wm[NV];
    TW qc = TW(0), qm = TW(0);
    TW da[NV], db[NV], dl[NV];
    const long long c = valid ? cidx(P, i, j, k) : 0;
    if (valid) {
        if constexpr (GLM) {
            const TW qa = (TW)Psi[c - st], qe = (TW)Psi[c + st];
            qc = (TW)Psi[c];
            const TW dq = limiter<TW>(P.limiter, qc - qa, qe - qc);
            qm = qc - TW(0.5) * dq;
            sQW[sl] = qc;
            sQP[sl] = qc + TW(0.5) * dq;
        }
        if (sizeof(TW) == 8 && sD) {
            // FP64: a cell's backward difference is its lower neighbour's forward difference; the
            // forward differences go through shared memory (the FP64 pipe is the bound, the load
            // / store path has room), and only the first cell of the tile subtracts its own
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const TW b = W[v * nt + c], e = W[v * nt + c + st];
                wc[v] = b;
                db[v] = e - b;
                sD[v * sz + sl] = db[v];
            }
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                TW a = W[v * nt + c - st], b = W[v * nt + c], e = W[v * nt + c + st];
                wc[v] = b;
                da[v] = b - a;
                db[v] = e - b;
            }
        }
    }
    if (sizeof(TW) == 8 && sD) {
        __syncthreads();                             // every thread: the forward differences are in sD
        if (valid) {
            const int pn = D == 0 ? sl - 1 : sl - BX;    // the neighbour one cell below along D
            if (ts > 0) {
#pragma unroll
                for (int v = 0; v < NV; ++v) da[v] = sD[v * sz + pn];
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v) da[v] = wc[v] - W[v * nt + c - st];
            }
        }
    }
    if (valid) {
        bool half = false;                       // dl holds half the limited slope
        if (P.limiter == 1 && sizeof(TW) == 8) {
            // FP64 van Leer 2ab/(a+b) for the eight fields with ONE division: batch inversion of
            // the eight sums (prefix products, one reciprocal, then peel off; zero sums replaced
            // by 1); the product stays far inside the double range unless all eight sums are
            // extreme, in which case the eight divisions are done one by one. dl = ab/(a+b), half
            // the slope: the factor 2 and the 1/2 of the face extrapolation cancel exactly
            half = true;
            TW s[NV], pre[NV];
            bool ok[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                s[v] = da[v] + db[v];
                ok[v] = ((hi_bits(da[v]) ^ hi_bits(db[v])) >= 0) && !is_zero(s[v]);
                if (!ok[v]) s[v] = TW(1);
            }
            pre[0] = s[0];
#pragma unroll
            for (int v = 1; v < NV; ++v) pre[v] = pre[v - 1] * s[v];
            const int ex = (hi_bits(pre[NV - 1]) >> 20) & 0x7ff;     // biased exponent of the product
            if (ex > 60 && ex < 1990) {
                TW inv = rcp_r(pre[NV - 1]);
#pragma unroll
                for (int v = NV - 1; v > 0; --v) {
                    const TW iv = inv * pre[v - 1];     // 1 / s[v]
                    inv = inv * s[v];                   // 1 / (s[0] ... s[v-1])
                    dl[v] = ok[v] ? da[v] * db[v] * iv : TW(0);
                }
                dl[0] = ok[0] ? da[0] * db[0] * inv : TW(0);
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v) dl[v] = ok[v] ? da[v] * db[v] / s[v] : TW(0);
            }
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) dl[v] = limiter<TW>(P.limiter, da[v], db[v]);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const TW h = half ? dl[v] : TW(0.5) * dl[v];
            wm[v] = wc[v] - h;
            sW[v * sz + sl] = wc[v];
            sP[v * sz + sl] = wc[v] + h;
        }
    }
    __syncthreads();
    if (valid && ts > 0 && s >= 0) {
        TW wl[NV], wr[NV], f[NV];
        const int pl = D == 0 ? sl - 1 : sl - BX;      // the neighbour one cell below along D
#pragma unroll
        for (int v = 0; v < NV; ++v) { wl[v] = sP[v * sz + pl]; wr[v] = wm[v]; }
        const bool first = not_positive(wl[0]) || not_positive(wr[0]) || not_positive(wl[4]) || not_positive(wr[4]);
        if (first) {
#pragma unroll
            for (int v = 0; v < NV; ++v) { wl[v] = sW[v * sz + pl]; wr[v] = wc[v]; }
        }
        riemann<TW, HD>(wl, wr, D, P.flux, phys<TW>(P).gamma, phys<TW>(P).igm1, f);
        long long fi, fs;
        if (D == 0) { fi = ((long long)k * P.n2 + j) * (P.n1 + 1) + s; fs = (long long)P.n3 * P.n2 * (P.n1 + 1); }
        else if (D == 1) { fi = ((long long)k * (P.n2 + 1) + s) * P.n1 + i; fs = (long long)P.n3 * (P.n2 + 1) * P.n1; }
        else { fi = ((long long)s * P.n2 + j) * P.n1 + i; fs = (long long)(P.n3 + 1) * P.n2 * P.n1; }
        if constexpr (GLM) {
            const TW sl_ = first ? sQW[pl] : sQP[pl], sr_ = first ? qc : qm;
            const TW bl = wl[5 + D], br = wr[5 + D];
            const double dt = P.sc->dt;         // 0 only for steps past a stop time (no change then)
            const TW ch = dt > 0.0 ? (TW)(P.sc->cfl * P.glm_dmin / dt) : TW(0);
            const TW bs = dt > 0.0 ? TW(0.5) * (bl + br) - TW(0.5) * (sr_ - sl_) / ch : TW(0.5) * (bl + br);
            f[5 + D] = TW(0.5) * (sl_ + sr_) - TW(0.5) * ch * (br - bl);
            FP[fi] = ch * ch * bs;
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v * fs + fi] = f[v];
    }
}

// number of tiles of a BX x BY flux tile along each launch axis
template <int D, int BX, int BY> __host__ __device__ inline void flux_tiles(const Params &P, int &nx, int &ny, int &nz)
{
    if (D == 0) { nx = (P.n1 + 1 + BX - 2) / (BX - 1); ny = (P.n2 + BY - 1) / BY; nz = P.n3; }
    else if (D == 1) { nx = (P.n1 + BX - 1) / BX; ny = (P.n2 + 1 + BY - 2) / (BY - 1); nz = P.n3; }
    else { nx = (P.n1 + BX - 1) / BX; ny = (P.n3 + 1 + BY - 2) / (BY - 1); nz = P.n2; }
}

template <int D> struct FluxShape {
    static constexpr int BX = D == 0 ? 128 : 16;
    static constexpr int BY = D == 0 ? 1 : 16;
};

// resident blocks per SM the TVDLF / HLL flux kernels are compiled for. FP64: at most 85 registers,
// so that 3 blocks of 256 threads (6 of 128) fit in the register file instead of 2 (5) at the 88
// the compiler takes unasked; the FP64 pipe is their bound, and more warps keep it busier. Single
// precision: at most 40 registers (6 blocks of 256, 12 of 128; a few bytes of spills) instead of
// 48, measured 3-7 % faster per flux kernel (issue-bound, latency-limited at 53-56 % warps
// active). No constraint for the HLLD instantiations.
template <int D, typename TW, bool HD> struct FluxMinBlocks {
    static constexpr int value = (sizeof(TW) == 8 && !HD) ? (D == 0 ? 6 : 3) : (!HD ? (D == 0 ? 12 : 6) : 1);
};

template <int D, typename TW, bool HD = false>
__global__ void __launch_bounds__(FluxShape<D>::BX * FluxShape<D>::BY, FluxMinBlocks<D, TW, HD>::value)
k_flux(Params P, const TW *__restrict__ W, TW *__restrict__ F)
{
    constexpr int BX = FluxShape<D>::BX, BY = FluxShape<D>::BY;
    __shared__ TW sW[NV * BY * BX];
    __shared__ TW sP[NV * BY * BX];
    __shared__ TW sD[sizeof(TW) == 8 && !HD ? NV * BY * BX : 1];   // FP64: forward differences
    flux_tile<D, BX, BY, TW, HD, false, TW>(P, W, F, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, threadIdx.y, sW,
                                            sP, nullptr, nullptr, nullptr, nullptr,
                                            sizeof(TW) == 8 && !HD ? sD : nullptr);
}

// the same with the GLM face step (psi of type TP, its face fluxes into FP)
template <int D, typename TW, bool HD, typename TP>
__global__ void __launch_bounds__(FluxShape<D>::BX * FluxShape<D>::BY)
k_flux_glm(Params P, const TW *__restrict__ W, TW *__restrict__ F, const TP *__restrict__ Psi, TW *__restrict__ FP)
{
    constexpr int BX = FluxShape<D>::BX, BY = FluxShape<D>::BY;
    __shared__ TW sW[NV * BY * BX];
    __shared__ TW sP[NV * BY * BX];
    __shared__ TW sQW[BY * BX];
    __shared__ TW sQP[BY * BX];
    flux_tile<D, BX, BY, TW, HD, true, TP>(P, W, F, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, threadIdx.y, sW, sP,
                                            Psi, FP, sQW, sQP);
}

// ---------------------------------------------------------------------------------------------
// div B at every cell of [-1, n]^3 from face averages of the cell-centred field
template <typename TW>
__device__ __forceinline__ void divb_cell(const Params &P, const TW *__restrict__ W, TW *__restrict__ divB, long long tid)
{
    const unsigned int e1 = P.n1 + 2, e2 = P.n2 + 2, ut = (unsigned int)tid;   // padded cells < 2^31
    const unsigned int r = ut / e1;
    const int i = (int)(ut - r * e1) - 1;
    const int j = (int)(r % e2) - 1;
    const int k = (int)(r / e2) - 1;
    const MetricsT<TW> &m = met<TW>(P);
    const long long nt = P.nt, c = cidx(P, i, j, k);
    const int ip = i + NG, jp = j + NG;
    const TW *b1 = W + 5 * nt, *b2 = W + 6 * nt, *b3 = W + 7 * nt;
    const long long s2 = P.p1, s3 = (long long)P.p1 * P.p2;
    TW d1, d2, d3;
    if constexpr (sizeof(TW) == 8) {
        // the face areas already divided by the volume factor (per-cell table); the halving on the
        // integer pipe
        d1 = cfv(m, CF_AP, ip, jp) * (b1[c] + b1[c + 1]) - cfv(m, CF_AM, ip, jp) * (b1[c - 1] + b1[c]);
        d2 = cfv(m, CF_BP, ip, jp) * (b2[c] + b2[c + s2]) - cfv(m, CF_BM, ip, jp) * (b2[c - s2] + b2[c]);
        d3 = (b3[c + s3] - b3[c - s3]) * cfv(m, CF_KV, ip, jp);
        divB[c] = half_r(d1 + d2 + d3);
    } else {
        d1 = (m.a1[ip + 1] * (b1[c] + b1[c + 1]) - m.a1[ip] * (b1[c - 1] + b1[c])) * m.iv1[ip];
        d2 = (m.a2[jp + 1] * (b2[c] + b2[c + s2]) - m.a2[jp] * (b2[c - s2] + b2[c])) * (m.q1[ip] * m.iv2[jp]);
        d3 = (b3[c + s3] - b3[c - s3]) * (m.q1[ip] * m.q2[jp] * m.iv3);
        divB[c] = TW(0.5) * (d1 + d2 + d3);
    }
}

template <typename TW>
__global__ void k_divb(Params P, const TW *__restrict__ W, TW *__restrict__ divB)
{
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)(P.n1 + 2) * (P.n2 + 2) * (P.n3 + 2)) return;
    divb_cell<TW>(P, W, divB, tid);
}

// ---------------------------------------------------------------------------------------------
// block-wide max and the last-block finalisation of dt
__device__ __forceinline__ double block_max(double v)
{
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    v = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;   // valid in thread 0
}

// advance_t: 1 after the second stage (t <- t + dt), 0 for a plain dt evaluation. Each block
// publishes its maximum with one 64-bit atomicMax on the bits of the double (for values > 0 the
// bit patterns order like the values; NaN, zeros and negatives are not published, as a maximum
// over the blocks starting from 0 with fmax, which drops NaN, would ignore them), and the block
// that arrives last reads the result: no pass over per-block partials after the grid
__device__ __forceinline__ void finish_dt(Params &P, double smax_block, int advance_t)
{
    __shared__ bool last;
    Scalars *sc = P.sc;
    if (threadIdx.x == 0) {
        if (smax_block > 0.0) atomicMax(&sc->smax_bits, (unsigned long long)__double_as_longlong(smax_block));
        __threadfence();
        unsigned int ticket = atomicAdd(&sc->done, 1u);
        last = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    const double v = __longlong_as_double((long long)*(volatile unsigned long long *)&sc->smax_bits);
    double t = sc->t;
    if (advance_t) t = __dadd_rn(t, sc->dt);
    double dt = sc->cfl / v;
    if (sc->t_stop > 0.0) dt = fmin(dt, fmax(__dsub_rn(sc->t_stop, t), 0.0));
    if (!(v > 0.0)) dt = 0.0;
    if (advance_t) sc->dt_step = sc->dt;
    sc->t = t;
    sc->dt = dt;
    sc->done = 0;
    sc->smax_bits = 0ull;
    sc->smax_seen = 0u;                 // every block of this launch has published its estimate
    // the step's status for icarus_step, which reads it on the host without synchronising
    if (advance_t && P.hstatus) *(volatile int *)P.hstatus = atomicOr(&sc->status, 0);
}

// CFL signal speed of one cell: sum_d (|v_d| + c_f,d) / dx_d, in the arithmetic type TW
template <typename TW>
__device__ __forceinline__ TW cell_speed_t(const Params &P, const TW *w, int ip, int jp)
{
    const MetricsT<TW> &m = met<TW>(P);
    TW irho = TW(1) / w[0];
    TW g = phys<TW>(P).gamma;
    TW s1 = (rabs(w[1]) + fast_speed<TW>(w, irho, 0, g)) * m.iw1[ip];
    TW s2 = (rabs(w[2]) + fast_speed<TW>(w, irho, 1, g)) * (m.ih2[ip] * m.id2);
    TW s3 = (rabs(w[3]) + fast_speed<TW>(w, irho, 2, g)) * (m.ih2[ip] * m.is3[jp] * m.id3);
    return s1 + s2 + s3;
}

template <typename TW>
__device__ __forceinline__ double cell_speed(const Params &P, const TW *w, int ip, int jp)
{
    return (double)cell_speed_t<TW>(P, w, ip, jp);
}

// double -> float by truncating the bit pattern, on the integer pipe (the FP64 pipe, which also
// carries conversions, is the scarce one): relative error below 2^-23 for 2^-126 <= |x| < 2^128,
// 0 below that range, +-FLT_MAX above it and for non-finite x
__device__ __forceinline__ float trunc_f(double x)
{
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int ax = hi & 0x7fffffff;
    const unsigned sign = (unsigned)hi & 0x80000000u;
    if (ax < 0x38100000) return 0.f;
    if (ax >= 0x47f00000) return __uint_as_float(sign | 0x7f7fffffu);
    return __uint_as_float(sign | ((unsigned)(ax - 0x38000000) << 3) | (lo >> 29));
}

// single-precision estimate of cell_speed from FP64 primitives. Its relative error stays below
// 1e-3: the fast-speed discriminant s^2 - 4 a^2 b_d^2 (s = a^2 + b^2) can cancel completely, so its
// absolute error is about 10 x 2^-24 s^2 (the roundings of s, s^2 and the product), which puts an
// error of at most sqrt(10 x 2^-24) / 2 = 4e-4 of s into c_f^2 >= s / 2, i.e. 4e-4 relative in c_f;
// the truncations add < 1e-6
__device__ __forceinline__ float cell_speed_est(const Params &P, const double *wd, int ip, int jp)
{
    const MetricsT<float> &m = P.mf;
    float w[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v] = trunc_f(wd[v]);
    const float irho = 1.f / w[0], g = P.phf.gamma, ih = m.ih2[ip];
    const float s1 = (fabsf(w[1]) + fast_speed<float>(w, irho, 0, g)) * m.iw1[ip];
    const float s2 = (fabsf(w[2]) + fast_speed<float>(w, irho, 1, g)) * (ih * m.id2);
    const float s3 = (fabsf(w[3]) + fast_speed<float>(w, irho, 2, g)) * (ih * m.is3[jp] * m.id3);
    return s1 + s2 + s3;
}

// block-wide max of a float, returned to every thread
__device__ __forceinline__ float block_max_all(float v)
{
    __shared__ float redf[33];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) redf[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < nw ? redf[lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) redf[32] = v;
    }
    __syncthreads();
    return redf[32];
}

// block maximum of the CFL signal speed (valid in thread 0; every thread of the block calls it).
// FP64: the single-precision estimate of every cell selects the cells within 1 % of the largest
// estimate seen, and only those evaluate the exact FP64 speed. With estimate errors below 1e-3
// the cell of the exact maximum always passes (its estimate is >= (1 - 1e-3) / (1 + 1e-3) of any
// cell's), so the result is the exact FP64 maximum, as if every cell had been evaluated. "Seen" is
// the block's own largest estimate, and, with glb (the launch's running maximum of the blocks'
// largest estimates as float bits, zero at the launch start), every earlier block's too: the blocks
// whose estimates all stay 1 % below one published by another block then evaluate no exact speed
template <typename TW>
__device__ __forceinline__ double cfl_block_speed(const Params &P, const TW *wo, int ip, int jp, bool valid,
                                                  unsigned int *glb = nullptr)
{
    if constexpr (sizeof(TW) == 4) {
        // single precision: reduce the float speeds, convert the block maximum once
        return (double)block_max_all(valid ? cell_speed_t<TW>(P, wo, ip, jp) : 0.f);
    } else {
        const float e = valid ? cell_speed_est(P, wo, ip, jp) : 0.f;
        float top = block_max_all(e);
        if (glb) {
            __shared__ float seen;
            if (threadIdx.x == 0) seen = fmaxf(top, __uint_as_float(atomicMax(glb, __float_as_uint(top))));
            __syncthreads();
            top = seen;
        }
        return block_max(valid && e >= top * 0.99f ? cell_speed<TW>(P, wo, ip, jp) : 0.0);
    }
}

template <typename TW>
__global__ void __launch_bounds__(256) k_cfl(Params P, const TW *__restrict__ W)
{
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (tid < (long long)P.n1 * P.n2 * P.n3) {
        int i = (int)(tid % P.n1);
        long long r = tid / P.n1;
        int j = (int)(r % P.n2), k = (int)(r / P.n2);
        long long c = cidx(P, i, j, k);
        TW w[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = W[v * P.nt + c];
        s = cell_speed<TW>(P, w, i + NG, j + NG);
    }
    s = block_max(s);
    finish_dt(P, s, 0);
}

// ---------------------------------------------------------------------------------------------
// conservative update of one stage:
//   L = -(1/V) sum_d (A+ F+ - A- F-) + S (geometric, rotating frame, gravity) ; Linde term
//   stage 1: U1 = U + dt L ; stage 2: U <- U/2 + (U1 + dt L)/2 ; floors ; primitives ; CFL (2)
// returns the cell's CFL signal speed after a second stage (0 otherwise)
// the update of one interior cell (i, j, k) from its primitives w, the fluxes through its six
// faces (lower / upper along r, theta, phi) and div B at its six neighbours; returns the cell's
// CFL signal speed after a second stage (0 otherwise)
// area / volume factors of the flux divergence of cell (i, j, k); in FP64 the area factors are
// multiplied by 1/V once per cell, so that a field costs one product and four fused
// multiply-adds on the FP64 pipe instead of three products and three
template <typename TW> struct DivFactors {
    TW am, ap, iv, bm, bp, jv, kv;
    __device__ __forceinline__ DivFactors(const MetricsT<TW> &m, int ip, int jp)
    {
        if constexpr (sizeof(TW) == 8) {
            // the products a1 iv1, a2 jv, kv from the per-cell table (loads instead of seven
            // products on the FP64 pipe; the same values)
            am = cfv(m, CF_AM, ip, jp); ap = cfv(m, CF_AP, ip, jp);
            bm = cfv(m, CF_BM, ip, jp); bp = cfv(m, CF_BP, ip, jp);
            kv = cfv(m, CF_KV, ip, jp);
            iv = jv = TW(0);
        } else {
            am = m.a1[ip]; ap = m.a1[ip + 1]; iv = m.iv1[ip]; bm = m.a2[jp]; bp = m.a2[jp + 1];
            jv = m.q1[ip] * m.iv2[jp];
            kv = m.q1[ip] * m.q2[jp] * m.iv3;
        }
    }
    // -(1/V) sum_d (A+ F+ - A- F-) of one field
    __device__ __forceinline__ TW div(TW fr0, TW fr1, TW ft0, TW ft1, TW fp0, TW fp1) const
    {
        if constexpr (sizeof(TW) == 8) {
            TW l = fma(am, fr0, -(ap * fr1));
            l = fma(bm, ft0, l);
            l = fma(-bp, ft1, l);
            return fma(-kv, fp1 - fp0, l);
        } else {
            TW l = -(ap * fr1 - am * fr0) * iv;
            l -= (bp * ft1 - bm * ft0) * jv;
            l -= (fp1 - fp0) * kv;
            return l;
        }
    }
};

// the update of one interior cell (i, j, k) from its primitives w, the flux divergence L (in:
// per field, out: the full residual), div B at its six neighbours, its stage-start state us(v)
// and (second stage) U^n un(v) (accessors, so that loads sit where they are used): the new state
// uo and primitives wo (floors applied and counted)
template <int STAGE, typename TS, typename TW, typename LS, typename LN>
__device__ __forceinline__ void update_math(const Params &P, int i, int j, int k, const TW *w, TW *L, const TW *dbn,
                                            LS us, LN un, TS *uo, TW *wo)
{
    const int ip = i + NG, jp = j + NG;
    const MetricsT<TW> &m = met<TW>(P);
    const PhysT<TW> &ph = phys<TW>(P);
    const double dt = P.sc->dt;
    if (P.geom == 0) {
        const TW rho = w[0], vr = w[1], vt = w[2], vp = w[3];
        const TW br = w[5], bt = w[6], bp = w[7];
        const TW ir = m.ih2[ip], cot = m.ct[jp];
        const TW pt = w[4] + half_r(br * br + bt * bt + bp * bp);
        // geometric terms of the spherical divergence; p_tot through face-area differences
        L[M1] += pt * m.gp1[ip] + (rho * (vt * vt + vp * vp) - (bt * bt + bp * bp)) * ir;
        const TW qg = sizeof(TW) == 8 ? cfv(m, CF_Q1GQ2, ip, jp) : m.q1[ip] * m.gq2[jp];
        L[M2] += pt * qg + (-(rho * vr * vt - br * bt) + cot * (rho * vp * vp - bp * bp)) * ir;
        L[M3] -= ((rho * vp * vr - bp * br) + cot * (rho * vp * vt - bp * bt)) * ir;
        L[B2] += (vr * bt - vt * br) * ir;
        L[B3] += ((vr * bp - vp * br) + cot * (vt * bp - vp * bt)) * ir;
        if (P.omega != 0.0) {
            // co-rotating frame, Omega along the polar axis: centrifugal rho Omega^2 r sin(th)
            // (sin th, cos th, 0), Coriolis 2 rho Omega (v_phi sin th, v_phi cos th,
            // -(v_r sin th + v_th cos th)), work of the centrifugal force in e
            const TW Om = ph.omega, sn = m.sn[jp], cs = m.cs[jp], rc = m.x1c[ip];
            const TW vpar = vr * sn + vt * cs;
            if constexpr (sizeof(TW) == 8) {
                // cen = (rho Omega) (Omega r sin th) with the second factor from the per-cell
                // table; the radial and polar parts share the bracket cen + 2 rho Omega v_phi
                const TW ro = rho * Om, ro2 = ro + ro;
                const TW cen = ro * cfv(m, CF_ORS, ip, jp);
                const TW t = cen + ro2 * vp;
                L[M1] += t * sn;
                L[M2] += t * cs;
                L[M3] -= ro2 * vpar;
                L[EN] += cen * vpar;
            } else {
                const TW cen = rho * Om * Om * rc * sn;
                L[M1] += cen * sn + TW(2) * rho * Om * vp * sn;
                L[M2] += cen * cs + TW(2) * rho * Om * vp * cs;
                L[M3] -= TW(2) * rho * Om * vpar;
                L[EN] += cen * vpar;
            }
        }
        if (P.gravity) {
            const TW g = m.gm_r2[ip];
            L[M1] -= rho * g;
            L[EN] -= rho * vr * g;
        }
    }
    // Powell's eight-wave source -(div B) (0, B, v.B, v) with the cell's own div B (dbn[6])
    if (P.divb == 3) {
        const TW d = dbn[6];
        L[M1] -= d * w[5]; L[M2] -= d * w[6]; L[M3] -= d * w[7];
        L[EN] -= d * (w[1] * w[5] + w[2] * w[6] + w[3] * w[7]);
        L[B1] -= d * w[1]; L[B2] -= d * w[2]; L[B3] -= d * w[3];
    }
    // Linde div-B diffusion: increment C_d / (sum_d 1/dx_d^2) grad(div B) per stage;
    // dbn = div B at (i-1, i+1, j-1, j+1, k-1, k+1)
    TW lb[3] = {TW(0), TW(0), TW(0)};
    if (P.divb == 1 && dt > 0.0) {
        if constexpr (sizeof(TW) == 8) {
            // coefficient times inverse widths from the per-cell table
            lb[0] = (dbn[1] - dbn[0]) * cfv(m, CF_LD0, ip, jp);
            lb[1] = (dbn[3] - dbn[2]) * cfv(m, CF_LD1, ip, jp);
            lb[2] = (dbn[5] - dbn[4]) * (cfv(m, CF_LD2, ip, jp) * m.ig3[k + NG]);
        } else {
            const TW coef = ph.divb_coef * m.ldx2[(long long)jp * P.p1 + ip];
            lb[0] = coef * (dbn[1] - dbn[0]) * m.ig1[ip];
            lb[1] = coef * (dbn[3] - dbn[2]) * (m.ih2[ip] * m.ig2[jp]);
            lb[2] = coef * (dbn[5] - dbn[4]) * (m.ih2[ip] * m.is3[jp] * m.ig3[k + NG]);
        }
    }
    if constexpr (Prec<TS, TW>::mixed) {
        // MIXED: the increment dt L + (Linde term) is formed in single precision like the fluxes it
        // comes from, and accumulated onto the FP64 state with one exact widening per field; the
        // second stage's average (U^n + U1 + increment) / 2 as in the FP64 form: two FP64 additions
        // and an exact halving on the integer pipe (the FP64 pipe bounds this kernel)
        const TW dtw = narrow_d2f(dt);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const TW inc = v >= B1 ? lb[v - B1] : (v == EN ? w[5] * lb[0] + w[6] * lb[1] + w[7] * lb[2] : TW(0));
            const TW d = dtw * L[v] + inc;
            const TS x = us(v) + widen_f2d(d);
            if (STAGE == 1) uo[v] = x;
            else uo[v] = half_r(un(v) + x);
        }
    } else {
        const TS dts = (TS)dt;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            // the Linde increment exists for e and B only (no addition of a zero for the others);
            // the second stage's average (U^n + x) / 2 with the halving on the integer pipe: the
            // same value as U^n / 2 + x / 2 (exact halvings, one rounding of the sum)
            TS x = us(v) + dts * (TS)L[v];
            if (v >= EN) x += (TS)(v >= B1 ? lb[v - B1] : w[5] * lb[0] + w[6] * lb[1] + w[7] * lb[2]);
            if (STAGE == 1) uo[v] = x;
            else uo[v] = half_r(un(v) + x);
        }
    }
    // non-finite check and floors
    bool bad = false;
#pragma unroll
    for (int v = 0; v < NV; ++v) bad |= (hi_bits(uo[v]) & (sizeof(TS) == 8 ? 0x7ff00000 : 0x7f800000)) ==
                                        (sizeof(TS) == 8 ? 0x7ff00000 : 0x7f800000);   // inf or NaN
    if (bad) atomicOr(&P.sc->status, 1);
    int hits = 0;
    const PhysT<TS> &phs = phys<TS>(P);
    if (uo[RHO] < phs.rho_floor) { uo[RHO] = phs.rho_floor; ++hits; }
    recover<TS, TW>(P, uo, wo, i);
    if (wo[4] < ph.p_floor) {
        // reset e so that p = p_floor, keeping rho, m, B
        TS ke = TS(0.5) * (uo[M1] * uo[M1] + uo[M2] * uo[M2] + uo[M3] * uo[M3]) / uo[RHO];
        TS me = TS(0.5) * (uo[B1] * uo[B1] + uo[B2] * uo[B2] + uo[B3] * uo[B3]);
        uo[EN] = phs.p_floor * phs.igm1 + ke + me;
        wo[4] = ph.p_floor;
        ++hits;
    }
    if (hits) {
        // one atomic per warp: the threads of the warp that hit a floor sum their counts first
        // (in a long run a large part of the grid can sit at the pressure floor, and one counter
        // taking an atomic from every such cell each stage serialises the update)
        const unsigned act = __activemask();
        const unsigned tot = __reduce_add_sync(act, (unsigned)hits);
        if ((int)(threadIdx.x & 31) == __ffs(act) - 1) {
            atomicAdd(&P.sc->floor_hits, (unsigned long long)tot);
            if (P.strict_floors) atomicOr(&P.sc->status, 2);
        }
    }
}

// update_math of cell (i, j, k) with its state read from and written to the global arrays (U^n is
// updated in place in the second stage)
template <int STAGE, typename TS, typename TW>
__device__ __forceinline__ void update_core(const Params &P, int i, int j, int k, const TW *w, TW *L, const TW *dbn,
                                            const TS *__restrict__ Us, TS *Uo, TW *__restrict__ Wo, TW *wo)
{
    const long long nt = P.nt, c = cidx(P, i, j, k);
    TS uo[NV];
    update_math<STAGE, TS, TW>(P, i, j, k, w, L, dbn, [&](int v) { return Us[v * nt + c]; },
                               [&](int v) { return Uo[v * nt + c]; }, uo, wo);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        Uo[v * nt + c] = uo[v];
        Wo[v * nt + c] = wo[v];
    }
}

// the update of cell number tid (r fastest) with fluxes and div B read from their global arrays;
// GLM: the flux form of grad psi leaves psi (A+ - A-) / V in the B_r and B_theta residuals
template <int STAGE, typename TS, typename TW, bool GLM = false>
__device__ __forceinline__ void update_cell(const Params &P, const TS *__restrict__ Us, const TW *__restrict__ Ws,
                                            TS *Uo, TW *__restrict__ Wo, const TW *__restrict__ F1,
                                            const TW *__restrict__ F2, const TW *__restrict__ F3,
                                            const TW *__restrict__ divB, long long tid, TW *wo)
{
    // interior cell numbers stay below 2^31 (the padded grid is limited to 2^31 cells): 32-bit
    // divisions instead of the 64-bit software sequence
    const unsigned int t32 = (unsigned int)tid, n1u = (unsigned int)P.n1, r_ = t32 / n1u;
    const int i = (int)(t32 - r_ * n1u);
    const int j = (int)(r_ % (unsigned int)P.n2), k = (int)(r_ / (unsigned int)P.n2);
    const long long nt = P.nt, c = cidx(P, i, j, k);
    TW w[NV], L[NV], dbn[7];
    const long long s1 = (long long)P.n3 * P.n2 * (P.n1 + 1), f1 = ((long long)k * P.n2 + j) * (P.n1 + 1) + i;
    const long long s2 = (long long)P.n3 * (P.n2 + 1) * P.n1, f2 = ((long long)k * (P.n2 + 1) + j) * P.n1 + i;
    const long long s3 = (long long)(P.n3 + 1) * P.n2 * P.n1, f3 = ((long long)k * P.n2 + j) * P.n1 + i;
    const long long o3 = (long long)P.n2 * P.n1;
    const DivFactors<TW> dv(met<TW>(P), i + NG, j + NG);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        w[v] = Ws[v * nt + c];
        L[v] = dv.div(F1[v * s1 + f1], F1[v * s1 + f1 + 1], F2[v * s2 + f2], F2[v * s2 + f2 + P.n1],
                      F3[v * s3 + f3], F3[v * s3 + f3 + o3]);
    }
    if (P.divb == 1) {
        const long long q2 = P.p1, q3 = (long long)P.p1 * P.p2;
        dbn[0] = divB[c - 1]; dbn[1] = divB[c + 1];
        dbn[2] = divB[c - q2]; dbn[3] = divB[c + q2];
        dbn[4] = divB[c - q3]; dbn[5] = divB[c + q3];
    } else if (P.divb == 3) {
        dbn[6] = divB[c];
    }
    if constexpr (GLM) {
        if (P.geom == 0) {
            const MetricsT<TW> &m = met<TW>(P);
            const TW psic = (TW)((const TS *)(STAGE == 1 ? P.psi0 : P.psi1))[c];
            L[B1] += psic * m.gp1[i + NG];
            L[B2] += psic * (m.q1[i + NG] * m.gq2[j + NG]);
        }
    }
    update_core<STAGE, TS, TW>(P, i, j, k, w, L, dbn, Us, Uo, Wo, wo);
}

template <int STAGE, typename TS, typename TW, bool GLM = false>
__device__ __forceinline__ void update_kernel_body(Params &P, const TS *__restrict__ Us, const TW *__restrict__ Ws, TS *Uo,
                                                   TW *__restrict__ Wo, const TW *__restrict__ F1,
                                                   const TW *__restrict__ F2, const TW *__restrict__ F3,
                                                   const TW *__restrict__ divB)
{
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = tid < (long long)P.n1 * P.n2 * P.n3;
    TW wo[NV];
    if (valid) update_cell<STAGE, TS, TW, GLM>(P, Us, Ws, Uo, Wo, F1, F2, F3, divB, tid, wo);
    if (STAGE == 2) {
        const unsigned int t32 = (unsigned int)tid, n1u = (unsigned int)P.n1;
        const int i = valid ? (int)(t32 % n1u) : 0, j = valid ? (int)((t32 / n1u) % (unsigned int)P.n2) : 0;
        finish_dt(P, cfl_block_speed<TW>(P, wo, i + NG, j + NG, valid, &P.sc->smax_seen), 1);
    }
}

template <int STAGE, typename TS, typename TW, bool GLM = false>
__global__ void __launch_bounds__(256)
k_update(Params P, const TS *__restrict__ Us, const TW *__restrict__ Ws, TS *Uo, TW *__restrict__ Wo,
         const TW *__restrict__ F1, const TW *__restrict__ F2, const TW *__restrict__ F3,
         const TW *__restrict__ divB)
{
    update_kernel_body<STAGE, TS, TW, GLM>(P, Us, Ws, Uo, Wo, F1, F2, F3, divB);
}

// the same update with at most 48 registers (5 blocks of 256 per SM): measured faster for the
// second MIXED stage, whose register demand otherwise limits it to 3 blocks
template <int STAGE, typename TS, typename TW>
__global__ void __launch_bounds__(256, 5)
k_update_capped(Params P, const TS *__restrict__ Us, const TW *__restrict__ Ws, TS *Uo, TW *__restrict__ Wo,
                const TW *__restrict__ F1, const TW *__restrict__ F2, const TW *__restrict__ F3,
                const TW *__restrict__ divB)
{
    update_kernel_body<STAGE, TS, TW>(P, Us, Ws, Uo, Wo, F1, F2, F3, divB);
}

// Cells per block of the update with the radial faces inside it (k_update_rf): a radial row of n1
// cells is cut into cdiv(n1, 128) segments of equal length, rounded up to whole warps; one block
// per segment
__host__ __device__ inline int rf_seg_cells(int n1)
{
    const int ns = (n1 + 127) / 128;
    return ((n1 + ns - 1) / ns + 31) / 32 * 32;
}
__host__ __device__ inline long long rf_blocks(const Params &P)
{
    const int c = rf_seg_cells(P.n1);
    return (long long)((P.n1 + c - 1) / c) * P.n2 * P.n3;
}

// The single-precision-flux update (TVDLF / HLL, Linde or Powell div B, no GLM) with the r-face
// fluxes of its radial row segment computed in the same kernel, so that they never go through
// HBM: the segment's primitives with a two-cell halo are staged in shared memory, each cell's
// limited slope and face states are formed once, each face's flux once, and every cell then takes
// its two r fluxes from shared memory and its theta / phi fluxes from the arrays of the separate
// flux kernels. The arithmetic of each step is that of flux_tile<0> and update_cell. Every
// thread of the block reaches the barriers (threads past the segment's end only skip the work).
// Measured at 512 x 64 x 128 (four segments of 128 per row, eight resident blocks per SM at 64
// registers): MIXED step 1.115 -> 1.012 ms, FP32 0.960 -> 0.877 ms against the r-flux kernel +
// update. Segments of 256 (four blocks per SM) took 1.050 / 0.896 ms, of 64 (sixteen) 1.035 /
// 0.927 ms; with 256, three or five resident blocks were slower than four
template <int STAGE, typename TS, typename TW>
__global__ void __launch_bounds__(128, 8)
k_update_rf(Params P, const TS *__restrict__ Us, const TW *__restrict__ Ws, TS *Uo, TW *__restrict__ Wo,
            const TW *__restrict__ F2, const TW *__restrict__ F3, const TW *__restrict__ divB)
{
    constexpr int CM = 128;
    __shared__ TW sW[NV][CM + 4];       // primitives of cells i0 - 2 .. i0 + nc + 1
    __shared__ TW sL[NV][CM + 2];       // lower-face states of cells i0 - 1 .. i0 + nc
    __shared__ TW sU[NV][CM + 2];       // upper-face states of the same cells
    __shared__ TW sF[NV][CM + 1];       // fluxes of r faces i0 .. i0 + nc (face i: cells i - 1, i)
    const int C = blockDim.x, t = threadIdx.x;
    const int ns = (P.n1 + C - 1) / C;
    const unsigned int row = blockIdx.x / (unsigned int)ns;
    const int seg = (int)(blockIdx.x - row * (unsigned int)ns);
    const int j = (int)(row % (unsigned int)P.n2), k = (int)(row / (unsigned int)P.n2);
    const int i0 = seg * C, nc = min(C, P.n1 - i0);
    const long long nt = P.nt, c0 = cidx(P, i0, j, k);
    for (int q = t; q < nc + 4; q += C) {
#pragma unroll
        for (int v = 0; v < NV; ++v) sW[v][q] = Ws[v * nt + c0 - 2 + q];
    }
    __syncthreads();
    for (int q = t; q < nc + 2; q += C) {          // cell i0 - 1 + q (sW index q + 1)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const TW wc = sW[v][q + 1];
            const TW h = TW(0.5) * limiter<TW>(P.limiter, wc - sW[v][q], sW[v][q + 2] - wc);
            sL[v][q] = wc - h;
            sU[v][q] = wc + h;
        }
    }
    __syncthreads();
    for (int f = t; f <= nc; f += C) {             // face i0 + f: slope index f below, f + 1 above
        TW wl[NV], wr[NV], fl[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) { wl[v] = sU[v][f]; wr[v] = sL[v][f + 1]; }
        if (not_positive(wl[0]) || not_positive(wr[0]) || not_positive(wl[4]) || not_positive(wr[4])) {
#pragma unroll
            for (int v = 0; v < NV; ++v) { wl[v] = sW[v][f + 1]; wr[v] = sW[v][f + 2]; }
        }
        riemann<TW, false>(wl, wr, 0, P.flux, phys<TW>(P).gamma, phys<TW>(P).igm1, fl);
#pragma unroll
        for (int v = 0; v < NV; ++v) sF[v][f] = fl[v];
    }
    __syncthreads();
    const bool valid = t < nc;
    const int i = i0 + t;
    TW wo[NV];
    if (valid) {
        const long long c = c0 + t;
        const long long s2 = (long long)P.n3 * (P.n2 + 1) * P.n1, f2 = ((long long)k * (P.n2 + 1) + j) * P.n1 + i;
        const long long s3 = (long long)(P.n3 + 1) * P.n2 * P.n1, f3 = ((long long)k * P.n2 + j) * P.n1 + i;
        const long long o3 = (long long)P.n2 * P.n1;
        const DivFactors<TW> dv(met<TW>(P), i + NG, j + NG);
        TW w[NV], L[NV], dbn[7];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            w[v] = sW[v][t + 2];
            L[v] = dv.div(sF[v][t], sF[v][t + 1], F2[v * s2 + f2], F2[v * s2 + f2 + P.n1], F3[v * s3 + f3],
                          F3[v * s3 + f3 + o3]);
        }
        if (P.divb == 1) {
            const long long q2 = P.p1, q3 = (long long)P.p1 * P.p2;
            dbn[0] = divB[c - 1]; dbn[1] = divB[c + 1];
            dbn[2] = divB[c - q2]; dbn[3] = divB[c + q2];
            dbn[4] = divB[c - q3]; dbn[5] = divB[c + q3];
        } else if (P.divb == 3) {
            dbn[6] = divB[c];
        }
        update_core<STAGE, TS, TW>(P, i, j, k, w, L, dbn, Us, Uo, Wo, wo);
    }
    if (STAGE == 2) finish_dt(P, cfl_block_speed<TW>(P, wo, (valid ? i : 0) + NG, j + NG, valid), 1);
}

// FP32 form, n1 even: one thread updates the two cells (i, i+1), i even, of a radial row with
// two-element vector loads and stores (every array offset of such a pair is even: p1, n1, the
// field strides and the base addresses are), which halves the memory instructions of this
// latency-bound kernel; the arithmetic is update_math per cell. (Measured on the MIXED form it was
// slower than one cell per thread: its FP64 state doubles the registers a pair needs.) Resident
// blocks per SM, measured at 512 x 64 x 128: the first stage at three (at most 85 registers, 0.176
// against 0.189 ms at two), the second, with U^n and the CFL reduction, at two (0.275 against 0.300
// ms at three)
template <typename T> struct Vec2;
template <> struct Vec2<float> { using t = float2; };
template <> struct Vec2<double> { using t = double2; };

template <int STAGE, typename TS, typename TW>
__global__ void __launch_bounds__(256, STAGE == 1 ? 3 : 2)
k_update_pair(Params P, const TS *__restrict__ Us, const TW *__restrict__ Ws, TS *Uo, TW *__restrict__ Wo,
              const TW *__restrict__ F1, const TW *__restrict__ F2, const TW *__restrict__ F3,
              const TW *__restrict__ divB)
{
    using S2 = typename Vec2<TS>::t;
    using W2 = typename Vec2<TW>::t;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int h = P.n1 / 2;
    const bool valid = tid < (long long)h * P.n2 * P.n3;
    TW wo[2][NV];
    int i = 0, j = 0;
    if (valid) {
        const unsigned int r_ = (unsigned int)tid / (unsigned int)h;
        i = 2 * (int)((unsigned int)tid - r_ * (unsigned int)h);
        j = (int)(r_ % (unsigned int)P.n2);
        const int k = (int)(r_ / (unsigned int)P.n2);
        const long long nt = P.nt, c = cidx(P, i, j, k);
        const long long s1 = (long long)P.n3 * P.n2 * (P.n1 + 1), f1 = ((long long)k * P.n2 + j) * (P.n1 + 1) + i;
        const long long s2 = (long long)P.n3 * (P.n2 + 1) * P.n1, f2 = ((long long)k * (P.n2 + 1) + j) * P.n1 + i;
        const long long s3 = (long long)(P.n3 + 1) * P.n2 * P.n1, f3 = ((long long)k * P.n2 + j) * P.n1 + i;
        const long long o3 = (long long)P.n2 * P.n1;
        const DivFactors<TW> dv0(met<TW>(P), i + NG, j + NG), dv1(met<TW>(P), i + 1 + NG, j + NG);
        TW w[2][NV], L[2][NV], dbn[2][7];
        TS us[2][NV], un[2][NV], uo[2][NV];
        (void)us; (void)un;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const W2 wv = *reinterpret_cast<const W2 *>(Ws + v * nt + c);
            w[0][v] = wv.x; w[1][v] = wv.y;
            const TW a0 = F1[v * s1 + f1], a1 = F1[v * s1 + f1 + 1], a2 = F1[v * s1 + f1 + 2];
            const W2 b0 = *reinterpret_cast<const W2 *>(F2 + v * s2 + f2);
            const W2 b1 = *reinterpret_cast<const W2 *>(F2 + v * s2 + f2 + P.n1);
            const W2 e0 = *reinterpret_cast<const W2 *>(F3 + v * s3 + f3);
            const W2 e1 = *reinterpret_cast<const W2 *>(F3 + v * s3 + f3 + o3);
            L[0][v] = dv0.div(a0, a1, b0.x, b1.x, e0.x, e1.x);
            L[1][v] = dv1.div(a1, a2, b0.y, b1.y, e0.y, e1.y);
            const S2 u2 = *reinterpret_cast<const S2 *>(Us + v * nt + c);
            us[0][v] = u2.x; us[1][v] = u2.y;
            if (STAGE == 2) {
                const S2 n2 = *reinterpret_cast<const S2 *>(Uo + v * nt + c);
                un[0][v] = n2.x; un[1][v] = n2.y;
            } else {
                un[0][v] = un[1][v] = TS(0);
            }
        }
        if (P.divb == 1) {
            const long long q2 = P.p1, q3 = (long long)P.p1 * P.p2;
            const W2 d0 = *reinterpret_cast<const W2 *>(divB + c);
            const W2 dm2 = *reinterpret_cast<const W2 *>(divB + c - q2), dp2 = *reinterpret_cast<const W2 *>(divB + c + q2);
            const W2 dm3 = *reinterpret_cast<const W2 *>(divB + c - q3), dp3 = *reinterpret_cast<const W2 *>(divB + c + q3);
            dbn[0][0] = divB[c - 1]; dbn[0][1] = d0.y; dbn[0][2] = dm2.x; dbn[0][3] = dp2.x; dbn[0][4] = dm3.x; dbn[0][5] = dp3.x;
            dbn[1][0] = d0.x; dbn[1][1] = divB[c + 2]; dbn[1][2] = dm2.y; dbn[1][3] = dp2.y; dbn[1][4] = dm3.y; dbn[1][5] = dp3.y;
        } else if (P.divb == 3) {
            const W2 d0 = *reinterpret_cast<const W2 *>(divB + c);
            dbn[0][6] = d0.x; dbn[1][6] = d0.y;
        }
        update_math<STAGE, TS, TW>(P, i, j, k, w[0], L[0], dbn[0], [&](int v) { return us[0][v]; },
                                   [&](int v) { return un[0][v]; }, uo[0], wo[0]);
        update_math<STAGE, TS, TW>(P, i + 1, j, k, w[1], L[1], dbn[1], [&](int v) { return us[1][v]; },
                                   [&](int v) { return un[1][v]; }, uo[1], wo[1]);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            S2 u2; u2.x = uo[0][v]; u2.y = uo[1][v];
            *reinterpret_cast<S2 *>(Uo + v * nt + c) = u2;
            W2 w2; w2.x = wo[0][v]; w2.y = wo[1][v];
            *reinterpret_cast<W2 *>(Wo + v * nt + c) = w2;
        }
    }
    if (STAGE == 2) {
        TW sp = TW(0);
        if (valid) sp = fmaxf(cell_speed_t<TW>(P, wo[0], i + NG, j + NG), cell_speed_t<TW>(P, wo[1], i + 1 + NG, j + NG));
        finish_dt(P, (double)block_max_all(sp), 1);
    }
}

// ---------------------------------------------------------------------------------------------
// GLM div-B control (Dedner et al. 2002). Along each face normal the pair (B_n, psi)
// obeys B_n,t + psi_n = 0, psi_t + c_h^2 B_n,n = 0; its exact upwind face state from the limited
// reconstructions (first order where the primitives fall back to it) gives B_n* and psi*: psi*
// replaces the normal-field flux of the MHD face flux, and psi is carried with flux c_h^2 B_n*.
// c_h = CFL dmin / dt (the fastest speed the step's dt carries over the smallest cell); after the
// second stage psi is damped by exp(-alpha c_h dt / dmin) = exp(-alpha CFL).
// Ghost values of psi along each direction at interior indices of the other two: copied like the
// MHD state, the driven face included (zero gradient).
template <typename TS>
__global__ void k_psi_ghost(Params P, TS *__restrict__ Psi)
{
    const long long nr = 2LL * NG * P.n2 * P.n3, nth = 2LL * NG * P.n1 * P.n3, nph = 2LL * NG * P.n1 * P.n2;
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nr + nth + nph) return;
    int D = 0;
    if (q >= nr) { q -= nr; D = 1; if (q >= nth) { q -= nth; D = 2; } }
    const int g = (int)(q % NG) + 1;
    long long r = q / NG;
    const int side = (int)(r % 2);
    r /= 2;
    const int n = D == 0 ? P.n1 : (D == 1 ? P.n2 : P.n3);
    const int na = D == 0 ? P.n2 : P.n1;
    const int a = (int)(r % na), b = (int)(r / na);
    const int gi = side == 0 ? -g : n - 1 + g;
    const int bc = P.bc[2 * D + side];
    auto at = [&](int s) -> long long {
        return D == 0 ? cidx(P, s, a, b) : (D == 1 ? cidx(P, a, s, b) : cidx(P, a, b, s));
    };
    // continuation and driven (1, 3), mirror (2), periodic (0)
    const int src = (bc == 1 || bc == 3) ? (side == 0 ? 0 : n - 1)
                  : (bc == 2 ? (side == 0 ? g - 1 : n - g) : ((gi % n) + n) % n);
    Psi[at(gi)] = Psi[at(src)];
}

// psi of every interior cell: stage 1 Psi1 = Psi + dt L; stage 2 Psi = (Psi/2 + (Psi1 + dt L)/2)
// damped (the second stage runs after the MHD update has advanced t and dt: the step's dt is
// dt_step)
template <int STAGE, typename TS, typename TW>
__global__ void k_glm_update(Params P, const TS *__restrict__ Ps, TS *Po, const TW *__restrict__ FP1,
                             const TW *__restrict__ FP2, const TW *__restrict__ FP3)
{
    const unsigned int tid = blockIdx.x * blockDim.x + threadIdx.x;   // cells < 2^31
    if (tid >= (unsigned int)(P.n1 * P.n2 * P.n3)) return;
    const unsigned int r_ = tid / (unsigned int)P.n1;
    const int i = (int)(tid - r_ * (unsigned int)P.n1), j = (int)(r_ % (unsigned int)P.n2),
              k = (int)(r_ / (unsigned int)P.n2);
    const long long c = cidx(P, i, j, k);
    const long long f1 = ((long long)k * P.n2 + j) * (P.n1 + 1) + i;
    const long long f2 = ((long long)k * (P.n2 + 1) + j) * P.n1 + i;
    const long long f3 = ((long long)k * P.n2 + j) * P.n1 + i;
    const DivFactors<TW> dv(met<TW>(P), i + NG, j + NG);
    const TW L = dv.div(FP1[f1], FP1[f1 + 1], FP2[f2], FP2[f2 + P.n1], FP3[f3], FP3[f3 + (long long)P.n2 * P.n1]);
    const double dt = STAGE == 1 ? P.sc->dt : P.sc->dt_step;
    if (STAGE == 1) Po[c] = Ps[c] + (TS)dt * (TS)L;
    else {
        const TS damp = dt > 0.0 ? (TS)exp(-P.glm_alpha * P.sc->cfl) : TS(1);
        Po[c] = (TS(0.5) * Po[c] + TS(0.5) * (Ps[c] + (TS)dt * (TS)L)) * damp;
    }
}

// psi of the interior from / to host-layout doubles [n3][n2][n1] (staged on the device)
template <typename TS>
__global__ void k_psi_copy(Params P, TS *Psi, double *buf, int to_psi)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)P.n1 * P.n2 * P.n3) return;
    const int i = (int)(tid % P.n1);
    const long long r_ = tid / P.n1;
    const int j = (int)(r_ % P.n2), k = (int)(r_ / P.n2);
    const long long c = cidx(P, i, j, k);
    if (to_psi) Psi[c] = (TS)buf[tid];
    else buf[tid] = (double)Psi[c];
}

// ---------------------------------------------------------------------------------------------
// CME tracer: a passive scalar c marking inserted CME plasma; rho c is conserved and carried by
// the mass flux with the limited linear reconstruction of c on the upwind side (so c = 1 moves
// exactly like rho); after each stage rho c is clipped to [0, rho].
// Ghost values of c for the cells the tracer stencil reads: the ghost layers along one direction
// at interior indices of the other two (its face fluxes never reach a corner). The driven face
// sets c = 1 in the CME footprint and 0 elsewhere; every other face copies like the MHD state.
template <typename TW>
__global__ void k_tracer_ghost(Params P, TW *__restrict__ C, int stage)
{
    const long long nr = 2LL * NG * P.n2 * P.n3, nth = 2LL * NG * P.n1 * P.n3, nph = 2LL * NG * P.n1 * P.n2;
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nr + nth + nph) return;
    int D = 0;
    if (q >= nr) { q -= nr; D = 1; if (q >= nth) { q -= nth; D = 2; } }
    const int g = (int)(q % NG) + 1;
    long long r = q / NG;
    const int side = (int)(r % 2);
    r /= 2;
    const int n = D == 0 ? P.n1 : (D == 1 ? P.n2 : P.n3);
    const int na = D == 0 ? P.n2 : P.n1;                 // first of the two other indices
    const int a = (int)(r % na), b = (int)(r / na);
    const int gi = side == 0 ? -g : n - 1 + g;
    const int bc = P.bc[2 * D + side];
    auto at = [&](int s) -> long long {
        return D == 0 ? cidx(P, s, a, b) : (D == 1 ? cidx(P, a, s, b) : cidx(P, a, b, s));
    };
    if (bc == 3) {                                      // driven (inner radial face)
        double tau = P.sc->t;
        if (stage == 2) tau = __dadd_rn(tau, P.sc->dt);
        double qq[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        C[at(gi)] = cme_column(P, tau, a, b, qq) ? TW(1) : TW(0);
        return;
    }
    // continuation (1), mirror (2), periodic (0)
    const int src = bc == 1 ? (side == 0 ? 0 : n - 1) : (bc == 2 ? (side == 0 ? g - 1 : n - g) : ((gi % n) + n) % n);
    C[at(gi)] = C[at(src)];
}

// limited slope of the tracer: van Leer branches around its division (c is zero, and its slopes
// vanish, in most of the domain); the other limiters as for the MHD variables
template <typename TW> __device__ __forceinline__ TW tracer_slope(int lim, TW a, TW b)
{
    if (lim != 1) return limiter<TW>(lim, a, b);
    if ((a > TW(0) && b > TW(0)) || (a < TW(0) && b < TW(0))) return TW(2) * a * b / (a + b);
    return TW(0);
}

template <int STAGE, typename TS, typename TW>
__global__ void __launch_bounds__(256)
k_tracer_update(Params P, const TW *__restrict__ C, const TW *__restrict__ F1, const TW *__restrict__ F2,
                const TW *__restrict__ F3, const TS *__restrict__ Ts, TS *To, const TS *__restrict__ Unew,
                TW *__restrict__ Cout)
{
    const unsigned int tid = blockIdx.x * blockDim.x + threadIdx.x;   // cells < 2^31
    if (tid >= (unsigned int)(P.n1 * P.n2 * P.n3)) return;
    const int i = (int)(tid % (unsigned int)P.n1);
    const unsigned int r_ = tid / (unsigned int)P.n1;
    const int j = (int)(r_ % (unsigned int)P.n2), k = (int)(r_ / (unsigned int)P.n2);
    const long long c = cidx(P, i, j, k);
    const long long f1 = ((long long)k * P.n2 + j) * (P.n1 + 1) + i;
    const long long f2 = ((long long)k * (P.n2 + 1) + j) * P.n1 + i;
    const long long f3 = ((long long)k * P.n2 + j) * P.n1 + i;
    const long long o3 = (long long)P.n2 * P.n1;
    const long long st[3] = {1, P.p1, (long long)P.p1 * P.p2};
    // tracer flux through the lower face of the cell at padded offset cb along d, with mass flux
    // fr: fr times the limited linear reconstruction of c on the upwind side (only that side)
    auto face = [&](int d, long long cb, TW fr) -> TW {
        const TW cm1 = C[cb - st[d]], c0 = C[cb];
        TW cu;
        if (fr >= TW(0)) cu = cm1 + TW(0.5) * tracer_slope<TW>(P.limiter, cm1 - C[cb - 2 * st[d]], c0 - cm1);
        else cu = c0 - TW(0.5) * tracer_slope<TW>(P.limiter, c0 - cm1, C[cb + st[d]] - c0);
        return fr * cu;
    };
    // density (field 0) fluxes: F1 [faces r], F2 [faces theta], F3 [faces phi]
    const TW r0 = face(0, c, F1[f1]), r1 = face(0, c + 1, F1[f1 + 1]);
    const TW t0 = face(1, c, F2[f2]), t1 = face(1, c + st[1], F2[f2 + P.n1]);
    const TW p0 = face(2, c, F3[f3]), p1 = face(2, c + st[2], F3[f3 + o3]);
    const DivFactors<TW> dv(met<TW>(P), i + NG, j + NG);
    const TW L = dv.div(r0, r1, t0, t1, p0, p1);
    const long long nt = P.nt;
    const double dt = STAGE == 1 ? P.sc->dt : P.sc->dt_step;   // the second stage's update has advanced t, dt
    TS to;
    if constexpr (Prec<TS, TW>::mixed) {
        const TW d = narrow_d2f(dt) * L + TW(0);
        if (STAGE == 1) to = Ts[c] + widen_f2d(d);
        else to = TS(0.5) * (To[c] + Ts[c]) + widen_f2d(TW(0.5) * d);
    } else {
        const TS dts = (TS)dt;
        if (STAGE == 1) to = Ts[c] + dts * (TS)L + (TS)TW(0);
        else to = TS(0.5) * To[c] + TS(0.5) * (Ts[c] + dts * (TS)L + (TS)TW(0));
    }
    const TS rho = Unew[RHO * nt + c];
    to = to < TS(0) ? TS(0) : (to > rho ? rho : to);
    To[c] = to;
    if constexpr (Prec<TS, TW>::mixed) Cout[c] = narrow_d2f(to) / narrow_d2f(rho);   // c in single precision
    else Cout[c] = (TW)(to / rho);
}

// rho c = rho * c_in from the current rho (c_in NULL: keep rho c); c = rho c / rho
template <typename TS, typename TW>
__global__ void k_tracer_set(Params P, const double *__restrict__ cin, const TS *__restrict__ U, TS *T, TW *C)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)P.n1 * P.n2 * P.n3) return;
    const int i = (int)(tid % P.n1);
    const long long r_ = tid / P.n1;
    const int j = (int)(r_ % P.n2), k = (int)(r_ / P.n2);
    const long long c = cidx(P, i, j, k);
    const TS rho = U[RHO * P.nt + c];
    if (cin) T[c] = (TS)((double)rho * cin[tid]);
    C[c] = (TW)(T[c] / rho);
}

template <typename TS>
__global__ void k_tracer_get(Params P, const TS *__restrict__ T, const TS *__restrict__ U, double *out)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)P.n1 * P.n2 * P.n3) return;
    const int i = (int)(tid % P.n1);
    const long long r_ = tid / P.n1;
    const int j = (int)(r_ % P.n2), k = (int)(r_ / P.n2);
    const long long c = cidx(P, i, j, k);
    out[tid] = (double)T[c] / (double)U[RHO * P.nt + c];
}

// ---------------------------------------------------------------------------------------------
// primitives of every padded cell (after a state upload)
template <typename TS, typename TW>
__global__ void k_prims(Params P, const TS *__restrict__ U, TW *__restrict__ W)
{
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.nt) return;
    int i = (int)(c % P.p1) - NG;
    TS u[NV];
    TW w[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = U[v * P.nt + c];
    if (u[RHO] == TS(0)) return;      // untouched ghost corner before the first fill
    recover<TS, TW>(P, u, w, i < 0 ? 0 : i);
#pragma unroll
    for (int v = 0; v < NV; ++v) W[v * P.nt + c] = w[v];
}

// initial state from the maps at the current time by radial expansion as a Parker wind:
// v_r const, rho ~ r^-2, p ~ r^-2 gamma, B_r ~ r^-2, B_phi = -B_r Omega r sin(theta) / v_r, and the
// flow radial in the inertial frame: v_phi = -Omega r sin(theta) in the co-rotating frame (the
// velocity is then parallel to the spiral field)
template <typename TS, typename TW>
__global__ void k_init_state(Params P, TS *__restrict__ U, TW *__restrict__ W, double r_in)
{
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)P.n1 * P.n2 * P.n3) return;
    int i = (int)(tid % P.n1);
    long long r_ = tid / P.n1;
    int j = (int)(r_ % P.n2), k = (int)(r_ / P.n2);
    double tau = P.sc->t;
    int m0 = 0, m1 = 0;
    double w = 0.0;
    int nm = P.n_maps;
    if (nm > 1 && tau > P.t_maps[0]) {
        if (tau >= P.t_maps[nm - 1]) m0 = m1 = nm - 1;
        else {
            int m = 0;
            while (m + 1 < nm - 1 && P.t_maps[m + 1] <= tau) ++m;
            m0 = m; m1 = m + 1;
            w = fmin(fmax((tau - P.t_maps[m]) / (P.t_maps[m + 1] - P.t_maps[m]), 0.0), 1.0);
        }
    }
    const long long per = (long long)P.n2 * P.n3, col = (long long)j * P.n3 + k;
    double b[5];
    for (int f = 0; f < 5; ++f)
        b[f] = (1.0 - w) * P.maps[((long long)m0 * 5 + f) * per + col] + w * P.maps[((long long)m1 * 5 + f) * per + col];
    const double r = P.m.x1c[i + NG], x = r_in / r, x2 = x * x;
    double wd[NV], ud[NV];
    wd[0] = b[1] * x2;
    wd[1] = b[0]; wd[2] = 0.0;
    wd[3] = P.init_vphi ? -P.omega * r * P.m.sn[j + NG] : 0.0;   // at rest co-rotating, or radial inertial flow
    wd[4] = b[2] * pow(x, 2.0 * P.gamma);
    wd[5] = b[3] * x2; wd[6] = 0.0;
    wd[7] = -wd[5] * P.omega * r * P.m.sn[j + NG] / wd[1];
    prim2cons<double>(wd, ud, 1.0 / (P.gamma - 1.0));
    long long c = cidx(P, i, j, k);
    TS us[NV];
    TW ws[NV];
    for (int v = 0; v < NV; ++v) us[v] = (TS)ud[v];
    recover<TS, TW>(P, us, ws, i);
    for (int v = 0; v < NV; ++v) {
        U[v * P.nt + c] = us[v];
        W[v * P.nt + c] = ws[v];
    }
}

// interior state <-> packed double array [8][n3][n2][n1]
template <typename TS>
__global__ void k_pack(Params P, const TS *__restrict__ U, double *__restrict__ out)
{
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long N = (long long)P.n1 * P.n2 * P.n3;
    if (tid >= N * NV) return;
    int v = (int)(tid / N);
    long long q = tid % N;
    int i = (int)(q % P.n1);
    long long r_ = q / P.n1;
    int j = (int)(r_ % P.n2), k = (int)(r_ / P.n2);
    out[tid] = (double)U[v * P.nt + cidx(P, i, j, k)];
}

template <typename TS>
__global__ void k_unpack(Params P, TS *__restrict__ U, const double *__restrict__ in)
{
    long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long N = (long long)P.n1 * P.n2 * P.n3;
    if (tid >= N * NV) return;
    int v = (int)(tid / N);
    long long q = tid % N;
    int i = (int)(q % P.n1);
    long long r_ = q / P.n1;
    int j = (int)(r_ % P.n2), k = (int)(r_ / P.n2);
    U[v * P.nt + cidx(P, i, j, k)] = (TS)in[tid];
}

// ---------------------------------------------------------------------------------------------
// probe sampling at the current time: one thread per probe, one block. Positions use only
// correctly rounded operations in a fixed order; the stencil is found by comparisons against
// the cell-centre arrays, so the indices do not depend on the arithmetic of the search.
template <typename TW>
__device__ __forceinline__ void probe_one(const Params &P, const TW *__restrict__ W, int p, long long head)
{
    Scalars *sc = P.sc;
    {
        const double AU = 1.495978707e11, PI = 3.14159265358979323846, TWO_PI = 2.0 * 3.14159265358979323846;
        const double tsi = __dmul_rn(sc->t, P.t0);
        const double *kn = P.traj + (long long)p * P.n_knots * 4;
        const int K = P.n_knots;
        int a = 0;
        double w = 0.0;
        if (K == 1 || tsi <= kn[0]) { a = 0; w = 0.0; }
        else if (tsi >= kn[(K - 1) * 4]) { a = K - 2; w = 1.0; }
        else {
            int lo = 0, hi = K - 1;              // largest a with kn[a] <= tsi, a <= K-2
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (kn[mid * 4] <= tsi) lo = mid; else hi = mid;
            }
            a = lo;
            w = __ddiv_rn(__dsub_rn(tsi, kn[a * 4]), __dsub_rn(kn[(a + 1) * 4], kn[a * 4]));
        }
        const int b = K == 1 ? 0 : a + 1;
        const double rm = __dadd_rn(kn[a * 4 + 1], __dmul_rn(w, __dsub_rn(kn[b * 4 + 1], kn[a * 4 + 1])));
        const double lat = __dadd_rn(kn[a * 4 + 2], __dmul_rn(w, __dsub_rn(kn[b * 4 + 2], kn[a * 4 + 2])));
        const double lon = __dadd_rn(kn[a * 4 + 3], __dmul_rn(w, __dsub_rn(kn[b * 4 + 3], kn[a * 4 + 3])));
        const double r = __ddiv_rn(rm, AU);
        const double th = __dsub_rn(PI / 2.0, lat);
        double ph = __dsub_rn(lon, __dmul_rn(P.omega_si, tsi));
        ph = __dsub_rn(ph, __dmul_rn(TWO_PI, floor(__ddiv_rn(ph, TWO_PI))));
        if (ph >= TWO_PI) ph = 0.0;
        const Metrics &m = P.m;
        const double *xc = m.x1c + NG, *yc = m.x2c + NG, *zc = m.x3c + NG;
        // r: estimate from the position, then move to the largest q in [0, n1-2] with xc[q] <= r
        int n1 = P.n1, n2 = P.n2, n3 = P.n3;
        int i = 0, j = 0, k;
        if (n1 > 1) {
            double est = (r - xc[0]) / (xc[1] - xc[0]);
            if (xc[1] / xc[0] > 1.0 + 1e-12 && P.geom == 0) est = log(r / xc[0]) / log(xc[1] / xc[0]);
            i = (int)fmin(fmax(floor(est), 0.0), (double)(n1 - 2));
            for (int it = 0; it < n1 && i < n1 - 2 && xc[i + 1] <= r; ++it) ++i;
            for (int it = 0; it < n1 && i > 0 && xc[i] > r; ++it) --i;
        }
        if (n2 > 1) {
            double est = (th - yc[0]) / (yc[1] - yc[0]);
            j = (int)fmin(fmax(floor(est), 0.0), (double)(n2 - 2));
            for (int it = 0; it < n2 && j < n2 - 2 && yc[j + 1] <= th; ++it) ++j;
            for (int it = 0; it < n2 && j > 0 && yc[j] > th; ++it) --j;
        }
        double phk;
        if (zc[0] > ph) { k = n3 - 1; phk = __dsub_rn(zc[n3 - 1], TWO_PI); }
        else {
            double est = floor((ph - zc[0]) * m.id3);
            k = (int)fmin(fmax(est, 0.0), (double)(n3 - 1));
            for (int it = 0; it < n3 && k < n3 - 1 && zc[k + 1] <= ph; ++it) ++k;
            for (int it = 0; it < n3 && k > 0 && zc[k] > ph; ++it) --k;
            phk = zc[k];
        }
        double wr = n1 > 1 ? (r - xc[i]) / (xc[i + 1] - xc[i]) : 0.0;
        double wt = n2 > 1 ? (th - yc[j]) / (yc[j + 1] - yc[j]) : 0.0;
        double wp = (ph - phk) * m.id3;
        wr = fmin(fmax(wr, 0.0), 1.0);
        wt = fmin(fmax(wt, 0.0), 1.0);
        wp = fmin(fmax(wp, 0.0), 1.0);
        const int i1 = n1 > 1 ? i + 1 : i, j1 = n2 > 1 ? j + 1 : j, k1 = (k + 1) % n3;
        double acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = 0.0;
        for (int cc = 0; cc < 8; ++cc) {
            int ci = (cc & 1) ? i1 : i, cj = (cc & 2) ? j1 : j, ck = (cc & 4) ? k1 : k;
            double f = ((cc & 1) ? wr : 1.0 - wr) * ((cc & 2) ? wt : 1.0 - wt) * ((cc & 4) ? wp : 1.0 - wp);
            long long c = cidx(P, ci, cj, ck);
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] += f * (double)W[v * P.nt + c];
        }
        const long long slot = head % P.ring_cap;
        double *q = P.ring + (slot * P.n_probes + p) * IC_NPROBE_REC;
        q[0] = tsi;
        q[1] = acc[0] * 1e6;
        q[2] = acc[1] * 1e5;
        q[3] = acc[2] * 1e5;
        q[4] = (acc[3] + P.omega * r * sin(th)) * 1e5;
        q[5] = acc[5] * P.b0;
        q[6] = acc[6] * P.b0;
        q[7] = acc[7] * P.b0;
        q[8] = acc[4] * P.p0;
        q[9] = sqrt(acc[5] * acc[5] + acc[6] * acc[6] + acc[7] * acc[7]) * P.b0;
        q[10] = i; q[11] = j; q[12] = k;
    }
}

template <typename TW>
__global__ void k_probe(Params P, const TW *__restrict__ W)
{
    const int p = threadIdx.x;
    const long long head = P.sc->ring_head;
    if (p < P.n_probes) probe_one<TW>(P, W, p, head);
    __syncthreads();
    if (p == 0) P.sc->ring_head = head + 1;
}

// ---------------------------------------------------------------------------------------------
// host-side launchers (one set per precision)
static inline unsigned int cdiv(long long a, long long b) { return (unsigned int)((a + b - 1) / b); }

template <typename TS, typename TW> struct Launch {
    static void fill_ghosts(const Params &P, void *U, void *W, int stage, cudaStream_t s)
    {
        TS *u = (TS *)U;
        TW *w = (TW *)W;
        const dim3 blk(64, 2 * NG);
        k_bnd1<TS, TW><<<dim3(cdiv(P.n2, 64), P.n3), blk, 0, s>>>(P, u, w, stage);
        k_bnd23<1, TS, TW><<<dim3(cdiv(P.p1, 64), P.n3), blk, 0, s>>>(P, u, w);
        k_bnd23<2, TS, TW><<<dim3(cdiv(P.p1, 64), P.p2), blk, 0, s>>>(P, u, w);
    }
    template <bool HD> static void flux_dir_t(const Params &P, int dir, const TW *w, TW *F, cudaStream_t s)
    {
        if (dir == 0) k_flux<0, TW, HD><<<dim3(cdiv(P.n1 + 1, 127), P.n2, P.n3), dim3(128, 1), 0, s>>>(P, w, F);
        else if (dir == 1) k_flux<1, TW, HD><<<dim3(cdiv(P.n1, 16), cdiv(P.n2 + 1, 15), P.n3), dim3(16, 16), 0, s>>>(P, w, F);
        else k_flux<2, TW, HD><<<dim3(cdiv(P.n1, 16), cdiv(P.n3 + 1, 15), P.n2), dim3(16, 16), 0, s>>>(P, w, F);
    }
    static void flux_dir(const Params &P, int dir, const void *W, void *F, cudaStream_t s)
    {
        if (P.flux == 2) flux_dir_t<true>(P, dir, (const TW *)W, (TW *)F, s);
        else flux_dir_t<false>(P, dir, (const TW *)W, (TW *)F, s);
    }
    static void fluxes(const Params &P, const void *W, void *F1, void *F2, void *F3, cudaStream_t s)
    {
        flux_dir(P, 0, W, F1, s);
        flux_dir(P, 1, W, F2, s);
        flux_dir(P, 2, W, F3, s);
    }
    static void divb(const Params &P, const void *W, void *D, cudaStream_t s)
    {
        long long n = (long long)(P.n1 + 2) * (P.n2 + 2) * (P.n3 + 2);
        k_divb<TW><<<cdiv(n, 256), 256, 0, s>>>(P, (const TW *)W, (TW *)D);
    }
    static void update(const Params &P, int stage, const void *Us, const void *Ws, void *Uo, void *Wo,
                       const void *F1, const void *F2, const void *F3, const void *D, cudaStream_t s)
    {
        long long n = (long long)P.n1 * P.n2 * P.n3;
        if constexpr (sizeof(TS) == 4 && sizeof(TW) == 4) if (P.n1 % 2 == 0 && P.divb != 2) {
            const long long np = n / 2;
            if (stage == 1)
                k_update_pair<1, TS, TW><<<cdiv(np, 256), 256, 0, s>>>(P, (const TS *)Us, (const TW *)Ws, (TS *)Uo,
                    (TW *)Wo, (const TW *)F1, (const TW *)F2, (const TW *)F3, (const TW *)D);
            else
                k_update_pair<2, TS, TW><<<cdiv(np, 256), 256, 0, s>>>(P, (const TS *)Us, (const TW *)Ws, (TS *)Uo,
                    (TW *)Wo, (const TW *)F1, (const TW *)F2, (const TW *)F3, (const TW *)D);
            return;
        }
        if (P.divb == 2) {                        // GLM: the plain update with the grad-psi terms
            if (stage == 1)
                k_update<1, TS, TW, true><<<cdiv(n, 256), 256, 0, s>>>(P, (const TS *)Us, (const TW *)Ws, (TS *)Uo,
                    (TW *)Wo, (const TW *)F1, (const TW *)F2, (const TW *)F3, (const TW *)D);
            else
                k_update<2, TS, TW, true><<<cdiv(n, 256), 256, 0, s>>>(P, (const TS *)Us, (const TW *)Ws, (TS *)Uo,
                    (TW *)Wo, (const TW *)F1, (const TW *)F2, (const TW *)F3, (const TW *)D);
            return;
        }
        if (stage == 1)
            k_update<1, TS, TW><<<cdiv(n, 256), 256, 0, s>>>(P, (const TS *)Us, (const TW *)Ws, (TS *)Uo, (TW *)Wo,
                (const TW *)F1, (const TW *)F2, (const TW *)F3, (const TW *)D);
        else if constexpr (Prec<TS, TW>::mixed)
            k_update_capped<2, TS, TW><<<cdiv(n, 256), 256, 0, s>>>(P, (const TS *)Us, (const TW *)Ws, (TS *)Uo,
                (TW *)Wo, (const TW *)F1, (const TW *)F2, (const TW *)F3, (const TW *)D);
        else
            k_update<2, TS, TW><<<cdiv(n, 256), 256, 0, s>>>(P, (const TS *)Us, (const TW *)Ws, (TS *)Uo, (TW *)Wo,
                (const TW *)F1, (const TW *)F2, (const TW *)F3, (const TW *)D);
    }
    // the update with the r faces inside it (replaces the r flux kernel and the update)
    static void update_rf(const Params &P, int stage, const void *Us, const void *Ws, void *Uo, void *Wo,
                          const void *F2, const void *F3, const void *D, cudaStream_t s)
    {
        const int c = rf_seg_cells(P.n1);
        const unsigned int nb = (unsigned int)rf_blocks(P);
        if (stage == 1)
            k_update_rf<1, TS, TW><<<nb, c, 0, s>>>(P, (const TS *)Us, (const TW *)Ws, (TS *)Uo, (TW *)Wo,
                (const TW *)F2, (const TW *)F3, (const TW *)D);
        else
            k_update_rf<2, TS, TW><<<nb, c, 0, s>>>(P, (const TS *)Us, (const TW *)Ws, (TS *)Uo, (TW *)Wo,
                (const TW *)F2, (const TW *)F3, (const TW *)D);
    }
    static void cfl(const Params &P, const void *W, cudaStream_t s)
    {
        long long n = (long long)P.n1 * P.n2 * P.n3;
        k_cfl<TW><<<cdiv(n, 256), 256, 0, s>>>(P, (const TW *)W);
    }
    static void probe(const Params &P, const void *W, cudaStream_t s)
    {
        k_probe<TW><<<1, ((P.n_probes + 31) / 32) * 32, 0, s>>>(P, (const TW *)W);
    }
    static void prims(const Params &P, const void *U, void *W, cudaStream_t s)
    {
        k_prims<TS, TW><<<cdiv(P.nt, 256), 256, 0, s>>>(P, (const TS *)U, (TW *)W);
    }
    static void init_state(const Params &P, void *U, void *W, double r_in, cudaStream_t s)
    {
        long long n = (long long)P.n1 * P.n2 * P.n3;
        k_init_state<TS, TW><<<cdiv(n, 256), 256, 0, s>>>(P, (TS *)U, (TW *)W, r_in);
    }
    static void pack(const Params &P, const void *U, double *out, cudaStream_t s)
    {
        long long n = (long long)P.n1 * P.n2 * P.n3 * NV;
        k_pack<TS><<<cdiv(n, 256), 256, 0, s>>>(P, (const TS *)U, out);
    }
    static void unpack(const Params &P, void *U, const double *in, cudaStream_t s)
    {
        long long n = (long long)P.n1 * P.n2 * P.n3 * NV;
        k_unpack<TS><<<cdiv(n, 256), 256, 0, s>>>(P, (TS *)U, in);
    }
    static void glm_ghost(const Params &P, void *Psi, cudaStream_t s)
    {
        const long long n = 2LL * NG * ((long long)P.n2 * P.n3 + (long long)P.n1 * P.n3 + (long long)P.n1 * P.n2);
        k_psi_ghost<TS><<<cdiv(n, 256), 256, 0, s>>>(P, (TS *)Psi);
    }
    template <bool HD>
    static void fluxes_glm_t(const Params &P, const TW *w, const TS *psi, TW *F1, TW *F2, TW *F3, TW *FP1, TW *FP2,
                             TW *FP3, cudaStream_t s)
    {
        k_flux_glm<0, TW, HD, TS><<<dim3(cdiv(P.n1 + 1, 127), P.n2, P.n3), dim3(128, 1), 0, s>>>(P, w, F1, psi, FP1);
        k_flux_glm<1, TW, HD, TS><<<dim3(cdiv(P.n1, 16), cdiv(P.n2 + 1, 15), P.n3), dim3(16, 16), 0, s>>>(P, w, F2, psi, FP2);
        k_flux_glm<2, TW, HD, TS><<<dim3(cdiv(P.n1, 16), cdiv(P.n3 + 1, 15), P.n2), dim3(16, 16), 0, s>>>(P, w, F3, psi, FP3);
    }
    // the three flux kernels with the GLM face step
    static void fluxes_glm(const Params &P, const void *W, const void *Psi, void *F1, void *F2, void *F3, void *FP1,
                           void *FP2, void *FP3, cudaStream_t s)
    {
        if (P.flux == 2)
            fluxes_glm_t<true>(P, (const TW *)W, (const TS *)Psi, (TW *)F1, (TW *)F2, (TW *)F3, (TW *)FP1, (TW *)FP2,
                               (TW *)FP3, s);
        else
            fluxes_glm_t<false>(P, (const TW *)W, (const TS *)Psi, (TW *)F1, (TW *)F2, (TW *)F3, (TW *)FP1, (TW *)FP2,
                                (TW *)FP3, s);
    }
    static void glm_update(const Params &P, int stage, const void *Ps, void *Po, const void *FP1, const void *FP2,
                           const void *FP3, cudaStream_t s)
    {
        const long long n = (long long)P.n1 * P.n2 * P.n3;
        if (stage == 1)
            k_glm_update<1, TS, TW><<<cdiv(n, 256), 256, 0, s>>>(P, (const TS *)Ps, (TS *)Po, (const TW *)FP1,
                (const TW *)FP2, (const TW *)FP3);
        else
            k_glm_update<2, TS, TW><<<cdiv(n, 256), 256, 0, s>>>(P, (const TS *)Ps, (TS *)Po, (const TW *)FP1,
                (const TW *)FP2, (const TW *)FP3);
    }
    static void psi_copy(const Params &P, void *Psi, double *buf, int to_psi, cudaStream_t s)
    {
        const long long n = (long long)P.n1 * P.n2 * P.n3;
        k_psi_copy<TS><<<cdiv(n, 256), 256, 0, s>>>(P, (TS *)Psi, buf, to_psi);
    }
    static void tracer_ghost(const Params &P, void *C, int stage, cudaStream_t s)
    {
        const long long n = 2LL * NG * ((long long)P.n2 * P.n3 + (long long)P.n1 * P.n3 + (long long)P.n1 * P.n2);
        k_tracer_ghost<TW><<<cdiv(n, 256), 256, 0, s>>>(P, (TW *)C, stage);
    }
    static void tracer_update(const Params &P, int stage, const void *C, const void *F1, const void *F2, const void *F3,
                              const void *Ts, void *To, const void *Unew, void *Cout, cudaStream_t s)
    {
        const long long n = (long long)P.n1 * P.n2 * P.n3;
        if (stage == 1)
            k_tracer_update<1, TS, TW><<<cdiv(n, 256), 256, 0, s>>>(P, (const TW *)C, (const TW *)F1, (const TW *)F2,
                (const TW *)F3, (const TS *)Ts, (TS *)To, (const TS *)Unew, (TW *)Cout);
        else
            k_tracer_update<2, TS, TW><<<cdiv(n, 256), 256, 0, s>>>(P, (const TW *)C, (const TW *)F1, (const TW *)F2,
                (const TW *)F3, (const TS *)Ts, (TS *)To, (const TS *)Unew, (TW *)Cout);
    }
    static void tracer_set(const Params &P, const double *cin, const void *U, void *T, void *C, cudaStream_t s)
    {
        const long long n = (long long)P.n1 * P.n2 * P.n3;
        k_tracer_set<TS, TW><<<cdiv(n, 256), 256, 0, s>>>(P, cin, (const TS *)U, (TS *)T, (TW *)C);
    }
    static void tracer_get(const Params &P, const void *T, const void *U, double *out, cudaStream_t s)
    {
        const long long n = (long long)P.n1 * P.n2 * P.n3;
        k_tracer_get<TS><<<cdiv(n, 256), 256, 0, s>>>(P, (const TS *)T, (const TS *)U, out);
    }
    static Ops make()
    {
        Ops o;
        o.fill_ghosts = fill_ghosts;
        o.fluxes = fluxes;
        o.flux_dir = flux_dir;
        o.divb = divb;
        o.update = update;
        o.cfl = cfl;
        o.probe = probe;
        o.prims = prims;
        o.init_state = init_state;
        o.pack = pack;
        o.unpack = unpack;
        o.fused_stage = nullptr;
        o.update_rf = nullptr;
        o.glm_ghost = glm_ghost;
        o.fluxes_glm = fluxes_glm;
        o.glm_update = glm_update;
        o.psi_copy = psi_copy;
        o.tracer_ghost = tracer_ghost;
        o.tracer_update = tracer_update;
        o.tracer_set = tracer_set;
        o.tracer_get = tracer_get;
        o.ts_size = sizeof(TS);
        o.tw_size = sizeof(TW);
        return o;
    }
};

}  // namespace icarus
