/*
 * icarus_oracle.c -- plain, slow FP64 CPU oracle of the Icarus 3.0 hot path (arXiv 2501.15923).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm may load this library. The CUDA library never calls it, and the
 * two share no code: this file defines its own constants, grid metrics and physics.
 *
 * What it computes, in the order of the method:
 *   - ideal MHD in conservative form with total pressure p_tot = p + B^2/2, mu0 = 1 (Sect. 2,
 *     Eqs. 1-6), gravity g = -GM/r^2 e_r (sign read as inward, see the note at gravity),
 *     co-rotating frame force F = rho (Omega x r) x Omega + 2 rho v x Omega and its work v.F
 *     (Sect. 2, Eqs. 2-3);
 *   - finite volumes on a spherical grid, radially stretched (dr ~ r) or uniform (Sect. 2, 3.2);
 *   - inner boundary at 0.1 AU from boundary maps interpolated linearly in time (Sect. 3), the
 *     same value in every ghost layer (Sect. 2.1), "asymm" for v_theta, v_phi, B_theta
 *     (Sect. 2.1), cone-CME overwrite inside the cone (Sect. 3.2, bc_icarus);
 *   - initial state from the first map by radial expansion (Sect. 2.1);
 *   - sampling along probe trajectories interpolated in time (Sect. 2).
 * The paper names no flux, limiter or integrator (it defers to the MPI-AMRVAC framework). This
 * oracle takes: limited linear reconstruction of primitives (minmod / van Leer / MC), TVDLF
 * (Rusanov) or HLL face flux, SSP-RK2 (Heun), two ghost layers, Linde-type div-B diffusion.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fast-math: every operation is an
 * IEEE double operation in source order).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- constants (SI) ------------------------------------------------------------------------ */
#define O_AU 1.495978707e11
#define O_MP 1.67262192369e-27
#define O_KB 1.380649e-23
#define O_MU0 1.25663706212e-6
#define O_GM 1.32712440018e20
#define O_PI 3.14159265358979323846

/* code units: L0 = 1 AU, v0 = 100 km/s, n0 = 1 cm^-3 (rho0 = m_p 1e6 kg/m^3), t0 = L0/v0,
 * p0 = rho0 v0^2, B0 = sqrt(mu0 rho0) v0 */
#define O_V0 1.0e5
#define O_N0 1.0e6

enum { RHO = 0, M1 = 1, M2 = 2, M3 = 3, EN = 4, B1 = 5, B2 = 6, B3 = 7, NV = 8 };
enum { BC_PERIODIC = 0, BC_CONT = 1, BC_REFLECT = 2, BC_DRIVEN = 3, BC_FIXED = 4 };
enum { GEOM_SPH = 0, GEOM_CART = 1 };
enum { LIM_MINMOD = 0, LIM_VANLEER = 1, LIM_MC = 2 };
enum { FLUX_TVDLF = 0, FLUX_HLL = 1, FLUX_HLLD = 2 };
enum { DIVB_NONE = 0, DIVB_LINDE = 1, DIVB_GLM = 2, DIVB_POWELL = 3 };

#define NG 2

typedef struct {
    int n[3], geom, stretch, bc[6];
    double xmin[3], xmax[3];
    int band_refine;                /* > 1: radial cells band_refine times narrower in [band_lo, band_hi] */
    double band_lo, band_hi;
    int p[3];
    long nt;                 /* padded cells */
    double *e[3];            /* edges, e[d][i+NG] = lower edge of cell i, i in [-NG, n+NG] */
    double *c[3];            /* centres, c[d][i+NG], i in [-NG, n+NG-1] */
    double gamma, omega_si, omega, gm;
    double cfl, divb_coef, rho_floor, p_floor;
    int limiter, flux, gravity, divb;
    int init_vphi;   /* initial v_phi: 0 at rest in the co-rotating frame, 1 inertially radial */
    int cme_model;   /* 0: cone footprint over a fixed window; 1: spherical cloud crossing r_in */
    double t0, p0, b0;       /* code-unit scales */
    double *U, *U0, *U1, *L, *W, *F[3], *divB, *Ufix;
    int tracer;                     /* CME tracer on: T = rho c, c = 1 in inserted CME plasma */
    /* GLM div-B control (divb = DIVB_GLM): psi and its stage copies (padded), the residual of
     * psi, the face fluxes of psi; c_h of the current step, the damping constant alpha, the
     * smallest cell width; Pcur = the psi the residual reads */
    double *Psi, *Psi0, *Psi1, *LPsi, *FP[3], *Pcur;
    double glm_alpha, glm_dmin, glm_ch;
    double *T, *T0, *T1, *LT, *C;   /* padded: rho c now / at the step start / stage 1, residual, c */
    double t;
    int n_maps; double *tm; double *maps;      /* code units, [n_maps][5][n2][n3] */
    int n_cme; double *cme;                    /* code units, [n_cme][8] */
    long floor_hits;
    int status;              /* 0 ok, 1 non-finite */
} orc_t;

#define IDX(o, i, j, k) ((((long)(k) + NG) * (o)->p[1] + ((j) + NG)) * (o)->p[0] + ((i) + NG))

/* ---- grid --------------------------------------------------------------------------------- */
/* Static refinement band (a fixed substitute for the paper's adaptive refinement, Sect. 2): in the
 * radial coordinate x (ln r on a stretched spherical grid, r or x otherwise) the cells are
 * band_refine times narrower inside [x(band_lo), x(band_hi)] than outside, with n1 cells over the
 * whole range: edge i sits where the cell-count density, 1 outside and band_refine inside,
 * integrates to i / n1 of its total. Ghost edges continue the outside spacing. */
static double band_edge(const orc_t *o, int i)
{
    const int lg = o->geom == GEOM_SPH && o->stretch;
    const double f = o->band_refine;
    const double X0 = lg ? log(o->xmin[0]) : o->xmin[0], X1 = lg ? log(o->xmax[0]) : o->xmax[0];
    const double A = lg ? log(o->band_lo) : o->band_lo, B = lg ? log(o->band_hi) : o->band_hi;
    if (i == 0) return o->xmin[0];
    if (i == o->n[0]) return o->xmax[0];
    const double total = (X1 - X0) + (f - 1.0) * (B - A);       /* integral of the density */
    const double s = total * i / o->n[0];
    const double sA = A - X0, sB = sA + f * (B - A);              /* the band's start and end in s */
    double x;
    if (s <= sA) x = X0 + s;
    else if (s <= sB) x = A + (s - sA) / f;
    else x = B + (s - sB);
    return lg ? exp(x) : x;
}

static double edge_pos(const orc_t *o, int d, int i)
{
    if (d == 0 && o->band_refine > 1) return band_edge(o, i);
    if (o->geom == GEOM_SPH && d == 0 && o->stretch)
        return o->xmin[0] * pow(o->xmax[0] / o->xmin[0], (double)i / o->n[0]);
    return o->xmin[d] + i * ((o->xmax[d] - o->xmin[d]) / o->n[d]);
}

static double lo(const orc_t *o, int d, int i) { return o->e[d][i + NG]; }
static double hi(const orc_t *o, int d, int i) { return o->e[d][i + NG + 1]; }
static double ctr(const orc_t *o, int d, int i) { return o->c[d][i + NG]; }

/* exact cell volume: (r+^3 - r-^3)/3 (cos th- - cos th+) dphi */
static double volume(const orc_t *o, int i, int j, int k)
{
    if (o->geom == GEOM_CART)
        return (hi(o, 0, i) - lo(o, 0, i)) * (hi(o, 1, j) - lo(o, 1, j)) * (hi(o, 2, k) - lo(o, 2, k));
    double rm = lo(o, 0, i), rp = hi(o, 0, i);
    return (rp * rp * rp - rm * rm * rm) / 3.0 * (cos(lo(o, 1, j)) - cos(hi(o, 1, j))) * (hi(o, 2, k) - lo(o, 2, k));
}

/* exact area of the LOWER face of cell (i,j,k) normal to direction d */
static double area(const orc_t *o, int d, int i, int j, int k)
{
    if (o->geom == GEOM_CART) {
        int a = (d + 1) % 3, b = (d + 2) % 3;
        int ia[3] = {i, j, k};
        return (hi(o, a, ia[a]) - lo(o, a, ia[a])) * (hi(o, b, ia[b]) - lo(o, b, ia[b]));
    }
    double rm = lo(o, 0, i), rp = hi(o, 0, i);
    double dph = hi(o, 2, k) - lo(o, 2, k);
    if (d == 0) return rm * rm * (cos(lo(o, 1, j)) - cos(hi(o, 1, j))) * dph;
    if (d == 1) return 0.5 * (rp * rp - rm * rm) * sin(lo(o, 1, j)) * dph;
    return 0.5 * (rp * rp - rm * rm) * (hi(o, 1, j) - lo(o, 1, j));
}

/* physical cell width along d (CFL and div-B coefficient) */
static double width(const orc_t *o, int d, int i, int j, int k)
{
    int ia[3] = {i, j, k};
    double w = hi(o, d, ia[d]) - lo(o, d, ia[d]);
    if (o->geom == GEOM_CART || d == 0) return w;
    if (d == 1) return ctr(o, 0, i) * w;
    return ctr(o, 0, i) * sin(ctr(o, 1, j)) * w;
}

/* ---- state conversions -------------------------------------------------------------------- */
static void cons2prim(const orc_t *o, const double *u, double *w)
{
    w[RHO] = u[RHO];
    w[1] = u[M1] / u[RHO];
    w[2] = u[M2] / u[RHO];
    w[3] = u[M3] / u[RHO];
    double ke = 0.5 * u[RHO] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
    double me = 0.5 * (u[B1] * u[B1] + u[B2] * u[B2] + u[B3] * u[B3]);
    w[4] = (o->gamma - 1.0) * (u[EN] - ke - me);
    w[5] = u[B1]; w[6] = u[B2]; w[7] = u[B3];
}

static void prim2cons(const orc_t *o, const double *w, double *u)
{
    u[RHO] = w[0];
    u[M1] = w[0] * w[1]; u[M2] = w[0] * w[2]; u[M3] = w[0] * w[3];
    u[EN] = w[4] / (o->gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3])
          + 0.5 * (w[5] * w[5] + w[6] * w[6] + w[7] * w[7]);
    u[B1] = w[5]; u[B2] = w[6]; u[B3] = w[7];
}

static void load(const orc_t *o, const double *A, long id, double *u)
{
    for (int v = 0; v < NV; v++) u[v] = A[v * o->nt + id];
}
static void store(const orc_t *o, double *A, long id, const double *u)
{
    for (int v = 0; v < NV; v++) A[v * o->nt + id] = u[v];
}

/* ---- physics: fast speed and fluxes (Eqs. 1-4 with p_tot of Eq. 6) ------------------------- */
/* c_f^2 = 1/2 (a^2 + b^2 + sqrt((a^2 + b^2)^2 - 4 a^2 B_d^2/rho)), a^2 = gamma p/rho, b^2 = B^2/rho */
static double fast_speed(const orc_t *o, const double *w, int d)
{
    double a2 = o->gamma * w[4] / w[0];
    double b2 = (w[5] * w[5] + w[6] * w[6] + w[7] * w[7]) / w[0];
    double bn2 = w[5 + d] * w[5 + d] / w[0];
    double s = a2 + b2;
    double disc = s * s - 4.0 * a2 * bn2;
    if (disc < 0.0) disc = 0.0;
    return sqrt(0.5 * (s + sqrt(disc)));
}

static void phys_flux(const orc_t *o, const double *w, const double *u, int d, double *f)
{
    double vn = w[1 + d], bn = w[5 + d];
    double bb = w[5] * w[5] + w[6] * w[6] + w[7] * w[7];
    double bv = w[5] * w[1] + w[6] * w[2] + w[7] * w[3];
    double ptot = w[4] + 0.5 * bb;
    f[RHO] = w[0] * vn;
    for (int c = 0; c < 3; c++) f[M1 + c] = w[0] * w[1 + c] * vn - w[5 + c] * bn;
    f[M1 + d] += ptot;
    f[EN] = (u[EN] + ptot) * vn - bn * bv;
    for (int c = 0; c < 3; c++) f[B1 + c] = vn * w[5 + c] - bn * w[1 + c];
}

static double limit(int lim, double a, double b)
{
    int same = (a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0);
    if (!same) return 0.0;
    if (lim == LIM_MINMOD) return fabs(a) < fabs(b) ? a : b;
    if (lim == LIM_VANLEER) return 2.0 * a * b / (a + b);
    /* monotonised central: sign * min(2|a|, 2|b|, |a+b|/2) */
    double m = fmin(fmin(2.0 * fabs(a), 2.0 * fabs(b)), 0.5 * fabs(a + b));
    return a > 0.0 ? m : -m;
}

/* HLLD (Miyoshi & Kusano 2005): four intermediate states separated by the entropy wave S_M and
 * the rotational waves S*_L, S*_R inside the fast waves S_L = min(u_L, u_R) - max(c_fL, c_fR),
 * S_R = max(u_L, u_R) + max(c_fL, c_fR). The normal field in the intermediate states is the mean
 * of the two face states. Where rho (S - u)(S - S_M) - B_n^2 vanishes (degenerate fast / Alfven
 * waves), the star state keeps the outer tangential velocity and field. */
static void hlld(const orc_t *o, const double *wl, const double *wr, int d, double *f)
{
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    double ul[NV], ur[NV], fl[NV], fr[NV];
    prim2cons(o, wl, ul);
    prim2cons(o, wr, ur);
    phys_flux(o, wl, ul, d, fl);
    phys_flux(o, wr, ur, d, fr);
    const double cl = fast_speed(o, wl, d), cr = fast_speed(o, wr, d);
    const double uL = wl[1 + d], uR = wr[1 + d];
    const double cmax = fmax(cl, cr);
    const double SL = fmin(uL, uR) - cmax, SR = fmax(uL, uR) + cmax;
    if (SL > 0.0) { for (int v = 0; v < NV; v++) f[v] = fl[v]; return; }
    if (SR < 0.0) { for (int v = 0; v < NV; v++) f[v] = fr[v]; return; }
    const double bn = 0.5 * (wl[5 + d] + wr[5 + d]);
    const double ptL = wl[4] + 0.5 * (wl[5] * wl[5] + wl[6] * wl[6] + wl[7] * wl[7]);
    const double ptR = wr[4] + 0.5 * (wr[5] * wr[5] + wr[6] * wr[6] + wr[7] * wr[7]);
    const double aL = (SL - uL) * wl[0], aR = (SR - uR) * wr[0];       /* mass fluxes relative to S */
    const double SM = (aR * uR - aL * uL - ptR + ptL) / (aR - aL);
    const double pts = (aR * ptL - aL * ptR + aL * aR * (uR - uL)) / (aR - aL);
    /* star states: index 0 left, 1 right */
    double us[2][NV], vt[2][2], bt[2][2], rs[2];
    for (int s = 0; s < 2; s++) {
        const double *w = s ? wr : wl, *u = s ? ur : ul;
        const double S = s ? SR : SL, a = s ? aR : aL, un = w[1 + d], pt = s ? ptR : ptL;
        const double rho = a / (S - SM);
        const double den = a * (S - SM) - bn * bn;
        const double scale = a * (S - un) + bn * bn;
        double vy = w[1 + t1], vz = w[1 + t2], by = w[5 + t1], bz = w[5 + t2];
        if (fabs(den) > 1e-12 * scale) {
            const double cv = bn * (SM - un) / den, cb = (a * (S - un) - bn * bn) / den;
            vy = w[1 + t1] - by * cv; vz = w[1 + t2] - bz * cv;
            by = w[5 + t1] * cb; bz = w[5 + t2] * cb;
        }
        const double vb = w[1] * w[5] + w[2] * w[6] + w[3] * w[7];
        const double vbs = SM * bn + vy * by + vz * bz;
        const double e = ((S - un) * u[EN] - pt * un + pts * SM + bn * (vb - vbs)) / (S - SM);
        rs[s] = rho;
        vt[s][0] = vy; vt[s][1] = vz; bt[s][0] = by; bt[s][1] = bz;
        us[s][RHO] = rho;
        us[s][M1 + d] = rho * SM; us[s][M1 + t1] = rho * vy; us[s][M1 + t2] = rho * vz;
        us[s][EN] = e;
        us[s][B1 + d] = bn; us[s][B1 + t1] = by; us[s][B1 + t2] = bz;
    }
    const double sqL = sqrt(rs[0]), sqR = sqrt(rs[1]);
    const double SsL = SM - fabs(bn) / sqL, SsR = SM + fabs(bn) / sqR;
    if (SsL >= 0.0) {                               /* F*_L */
        for (int v = 0; v < NV; v++) f[v] = fl[v] + SL * (us[0][v] - ul[v]);
        return;
    }
    if (SsR <= 0.0) {                               /* F*_R */
        for (int v = 0; v < NV; v++) f[v] = fr[v] + SR * (us[1][v] - ur[v]);
        return;
    }
    /* double-star states (shared tangential velocity and field) */
    const double sg = bn > 0.0 ? 1.0 : (bn < 0.0 ? -1.0 : 0.0), isum = 1.0 / (sqL + sqR);
    double vss[2], bss[2];
    for (int c = 0; c < 2; c++) {
        vss[c] = (sqL * vt[0][c] + sqR * vt[1][c] + (bt[1][c] - bt[0][c]) * sg) * isum;
        bss[c] = (sqL * bt[1][c] + sqR * bt[0][c] + sqL * sqR * (vt[1][c] - vt[0][c]) * sg) * isum;
    }
    const double vbss = SM * bn + vss[0] * bss[0] + vss[1] * bss[1];
    const int s = SM >= 0.0 ? 0 : 1;                /* side of the entropy wave */
    const double sq = s ? sqR : sqL, Ss = s ? SsR : SsL, S = s ? SR : SL;
    const double *uo = s ? ur : ul, *fo = s ? fr : fl;
    const double vbs = SM * bn + vt[s][0] * bt[s][0] + vt[s][1] * bt[s][1];
    double uss[NV];
    uss[RHO] = rs[s];
    uss[M1 + d] = rs[s] * SM; uss[M1 + t1] = rs[s] * vss[0]; uss[M1 + t2] = rs[s] * vss[1];
    uss[EN] = us[s][EN] + (s ? 1.0 : -1.0) * sq * (vbs - vbss) * sg;
    uss[B1 + d] = bn; uss[B1 + t1] = bss[0]; uss[B1 + t2] = bss[1];
    for (int v = 0; v < NV; v++) f[v] = fo[v] + S * (us[s][v] - uo[v]) + Ss * (uss[v] - us[s][v]);
}

/* TVDLF: F = (F_L + F_R)/2 - c_max (U_R - U_L)/2, c_max = max(|v_n| + c_f) over L and R.
 * HLL:   F = (s_R F_L - s_L F_R + s_L s_R (U_R - U_L)) / (s_R - s_L), upwinded outside the fan.
 * HLLD:  see hlld(). */
static void riemann(const orc_t *o, const double *wl, const double *wr, int d, double *f)
{
    if (o->flux == FLUX_HLLD) { hlld(o, wl, wr, d, f); return; }
    double ul[NV], ur[NV], fl[NV], fr[NV];
    prim2cons(o, wl, ul);
    prim2cons(o, wr, ur);
    phys_flux(o, wl, ul, d, fl);
    phys_flux(o, wr, ur, d, fr);
    double cl = fast_speed(o, wl, d), cr = fast_speed(o, wr, d);
    if (o->flux == FLUX_TVDLF) {
        double c = fmax(fabs(wl[1 + d]) + cl, fabs(wr[1 + d]) + cr);
        for (int v = 0; v < NV; v++) f[v] = 0.5 * (fl[v] + fr[v]) - 0.5 * c * (ur[v] - ul[v]);
    } else {
        double sl = fmin(wl[1 + d] - cl, wr[1 + d] - cr);
        double sr = fmax(wl[1 + d] + cl, wr[1 + d] + cr);
        if (sl >= 0.0) { for (int v = 0; v < NV; v++) f[v] = fl[v]; return; }
        if (sr <= 0.0) { for (int v = 0; v < NV; v++) f[v] = fr[v]; return; }
        for (int v = 0; v < NV; v++)
            f[v] = (sr * fl[v] - sl * fr[v] + sl * sr * (ur[v] - ul[v])) / (sr - sl);
    }
}

/* ---- boundary conditions ------------------------------------------------------------------ */
static void copy_cell(orc_t *o, double *U, long dst, long src, int flip_d)
{
    for (int v = 0; v < NV; v++) U[v * o->nt + dst] = U[v * o->nt + src];
    if (flip_d >= 0) {
        U[(M1 + flip_d) * o->nt + dst] = -U[(M1 + flip_d) * o->nt + dst];
        U[(B1 + flip_d) * o->nt + dst] = -U[(B1 + flip_d) * o->nt + dst];
    }
}

static long cell_id(const orc_t *o, int d, int g, int a, int b)
{
    /* cell whose index along d is g and whose other two indices are (a, b) in cyclic order */
    int ia[3];
    ia[d] = g; ia[(d + 1) % 3] = a; ia[(d + 2) % 3] = b;
    return IDX(o, ia[0], ia[1], ia[2]);
}

/* linear time interpolation of the boundary maps (Sect. 3): bracket tau between consecutive map
 * times, weight w in [0, 1], clamp to the first / last map outside the table */
static void map_bracket(const orc_t *o, double tau, int *m0, int *m1, double *w)
{
    int n = o->n_maps;
    if (n == 1 || tau <= o->tm[0]) { *m0 = *m1 = 0; *w = 0.0; return; }
    if (tau >= o->tm[n - 1]) { *m0 = *m1 = n - 1; *w = 0.0; return; }
    int m = 0;
    while (m + 1 < n - 1 && o->tm[m + 1] <= tau) m++;
    *m0 = m; *m1 = m + 1;
    double ww = (tau - o->tm[m]) / (o->tm[m + 1] - o->tm[m]);
    if (ww < 0.0) ww = 0.0;
    if (ww > 1.0) ww = 1.0;
    *w = ww;
}

/* map primitives (rho, v_r, p, B_r, B_phi) at column (j,k) and time tau, before any CME */
static void map_value(const orc_t *o, double tau, int j, int k, double *out5)
{
    int m0, m1; double w;
    map_bracket(o, tau, &m0, &m1, &w);
    int n2 = o->n[1], n3 = o->n[2];
    for (int f = 0; f < 5; f++) {
        double a = o->maps[(((long)m0 * 5 + f) * n2 + j) * n3 + k];
        double b = o->maps[(((long)m1 * 5 + f) * n2 + j) * n3 + k];
        out5[f] = (1.0 - w) * a + w * b;
    }
}

/* cone CME (Sect. 3.2): a boundary column lies in the CME when the angle alpha between its
 * centre direction and the CME axis is small enough; the test compares the dot product of the two
 * unit vectors, cos(alpha), with a threshold. Model 0: the cone of the half-width omega over the
 * window [t_on, t_on + duration): threshold cos(omega). Model 1: a spherical cloud of radius
 * R = r_in sin(omega) whose centre moves out along the axis at the CME speed v, its leading point
 * reaching r_in at t_on (centre distance d = r_in - R + v (tau - t_on)); a column at r_in is inside
 * while |r_in e - d a| <= R, i.e. cos(alpha) >= (r_in^2 + d^2 - R^2) / (2 r_in d), for
 * tau in [t_on, t_on + 2 R / v) (the duration entry is not used). Later CMEs override earlier ones. */
static int cme_hit(const orc_t *o, double tau, int j, int k, double *out5)
{
    int hit = 0;
    double th = ctr(o, 1, j), ph = ctr(o, 2, k);
    double ex = sin(th) * cos(ph), ey = sin(th) * sin(ph), ez = cos(th);
    for (int c = 0; c < o->n_cme; c++) {
        const double *q = o->cme + 8 * c;
        double thr = cos(q[4]);
        if (o->cme_model == 1) {
            double rb = o->xmin[0], R = rb * sin(q[4]);
            if (!(tau >= q[0] && tau < q[0] + 2.0 * R / q[5])) continue;
            double d = (rb - R) + q[5] * (tau - q[0]);
            thr = (rb * rb + d * d - R * R) / (2.0 * rb * d);
        } else if (!(tau >= q[0] && tau < q[0] + q[1])) {
            continue;
        }
        double lat = q[2], lon = q[3];
        double ax = cos(lat) * cos(lon), ay = cos(lat) * sin(lon), az = sin(lat);
        double dot = ex * ax + ey * ay + ez * az;
        if (dot >= thr) {
            out5[0] = q[6];   /* rho (code) */
            out5[1] = q[5];   /* v_r */
            out5[2] = q[7];   /* p */
            hit = 1;
        }
    }
    return hit;
}

static void driven_fill(orc_t *o, double *U, double tau)
{
    if (o->n_maps < 1) return;
    for (int k = 0; k < o->n[2]; k++)
        for (int j = 0; j < o->n[1]; j++) {
            double b[5];
            map_value(o, tau, j, k, b);
            /* map order is (v_r, n, p, B_r, B_phi); reorder to (rho, v_r, p, B_r, B_phi) */
            double q[5] = {b[1], b[0], b[2], b[3], b[4]};
            cme_hit(o, tau, j, k, q);
            for (int g = 1; g <= NG; g++) {
                double um[NV], wm[NV], w[NV], u[NV];
                load(o, U, IDX(o, g - 1, j, k), um);
                cons2prim(o, um, wm);
                w[0] = q[0]; w[1] = q[1]; w[4] = q[2]; w[5] = q[3]; w[7] = q[4];
                w[2] = -wm[2]; w[3] = -wm[3]; w[6] = -wm[6];      /* asymm */
                prim2cons(o, w, u);
                store(o, U, IDX(o, -g, j, k), u);
            }
        }
}

static void fill_side(orc_t *o, double *U, int d, int side, double tau)
{
    int bc = o->bc[2 * d + side];
    int n = o->n[d];
    int a_lo = -NG, a_hi = o->n[(d + 1) % 3] + NG, b_lo = -NG, b_hi = o->n[(d + 2) % 3] + NG;
    /* r ghosts: interior (theta, phi) only; theta ghosts: every r incl. ghosts, interior phi;
     * phi ghosts: everything. This fixes the corner values. */
    if (d == 0) { a_lo = 0; a_hi = o->n[1]; b_lo = 0; b_hi = o->n[2]; }
    if (d == 1) { a_lo = 0; a_hi = o->n[2]; b_lo = -NG; b_hi = o->n[0] + NG; }
    if (bc == BC_DRIVEN) { driven_fill(o, U, tau); return; }
    for (int b = b_lo; b < b_hi; b++)
        for (int a = a_lo; a < a_hi; a++)
            for (int g = 1; g <= NG; g++) {
                int gi = side == 0 ? -g : n - 1 + g;
                int src, flip = -1;
                if (bc == BC_CONT) src = side == 0 ? 0 : n - 1;
                else if (bc == BC_REFLECT) { src = side == 0 ? g - 1 : n - g; flip = d; }
                else if (bc == BC_PERIODIC) src = ((gi % n) + n) % n;
                else { /* FIXED: keep the values captured at set-state time */
                    long id = cell_id(o, d, gi, a, b);
                    for (int v = 0; v < NV; v++) U[v * o->nt + id] = o->Ufix[v * o->nt + id];
                    continue;
                }
                copy_cell(o, U, cell_id(o, d, gi, a, b), cell_id(o, d, src, a, b), flip);
                if (d == 0 && side == 1 && bc == BC_CONT && o->geom == GEOM_SPH) {
                    /* outer radius: B_r continues as r^-2 (the radial flux r^2 B_r is what is
                     * copied), so the ghost layer adds no divergence; e follows the change of B^2 */
                    long id = cell_id(o, d, gi, a, b);
                    double f = (ctr(o, 0, src) / ctr(o, 0, gi)) * (ctr(o, 0, src) / ctr(o, 0, gi));
                    double bs = U[B1 * o->nt + id], bg = bs * f;
                    U[EN * o->nt + id] += 0.5 * (bg * bg - bs * bs);
                    U[B1 * o->nt + id] = bg;
                }
            }
}

static void fill_ghosts(orc_t *o, double *U, double tau)
{
    fill_side(o, U, 0, 0, tau);
    fill_side(o, U, 0, 1, tau);
    fill_side(o, U, 1, 0, tau);
    fill_side(o, U, 1, 1, tau);
    fill_side(o, U, 2, 0, tau);
    fill_side(o, U, 2, 1, tau);
}

/* ---- residual L(U) ------------------------------------------------------------------------ */
static void all_prims(orc_t *o, const double *U)
{
#pragma omp parallel for
    for (long id = 0; id < o->nt; id++) {
        double u[NV], w[NV];
        load(o, U, id, u);
        cons2prim(o, u, w);
        store(o, o->W, id, w);
    }
}

/* flux through the lower face (along d) of every cell (i,j,k) with index along d in [0, n_d] */
static void face_fluxes(orc_t *o, int d)
{
    int ext[3] = {o->n[0], o->n[1], o->n[2]};
    ext[d] += 1;
    int sh[3] = {0, 0, 0};
    sh[d] = 1;
#pragma omp parallel for collapse(2)
    for (int k = 0; k < ext[2]; k++)
        for (int j = 0; j < ext[1]; j++)
            for (int i = 0; i < ext[0]; i++) {
                double wm2[NV], wm1[NV], w0[NV], wp1[NV], wl[NV], wr[NV], f[NV];
                /* cells b-2, b-1 (= a), b, b+1 along d, with b the cell (i,j,k) */
                load(o, o->W, IDX(o, i - 2 * sh[0], j - 2 * sh[1], k - 2 * sh[2]), wm2);
                load(o, o->W, IDX(o, i - sh[0], j - sh[1], k - sh[2]), wm1);
                load(o, o->W, IDX(o, i, j, k), w0);
                load(o, o->W, IDX(o, i + sh[0], j + sh[1], k + sh[2]), wp1);
                for (int v = 0; v < NV; v++) {
                    double da = limit(o->limiter, wm1[v] - wm2[v], w0[v] - wm1[v]);
                    double db = limit(o->limiter, w0[v] - wm1[v], wp1[v] - w0[v]);
                    wl[v] = wm1[v] + 0.5 * da;
                    wr[v] = w0[v] - 0.5 * db;
                }
                const int first = wl[0] <= 0.0 || wr[0] <= 0.0 || wl[4] <= 0.0 || wr[4] <= 0.0;
                if (first)
                    for (int v = 0; v < NV; v++) { wl[v] = wm1[v]; wr[v] = w0[v]; }
                riemann(o, wl, wr, d, f);
                if (o->divb == DIVB_GLM) {
                    /* GLM (Dedner et al. 2002): the (B_n, psi) pair obeys B_n,t + psi_n = 0,
                     * psi_t + c_h^2 B_n,n = 0 along the normal; its exact upwind face state replaces
                     * the normal-field flux by psi* and gives psi the flux c_h^2 B_n*. psi is
                     * reconstructed like the primitives (first order where they are). */
                    const double *P = o->Pcur;
                    long ib = IDX(o, i, j, k), s1 = IDX(o, i - sh[0], j - sh[1], k - sh[2]);
                    long s2 = IDX(o, i - 2 * sh[0], j - 2 * sh[1], k - 2 * sh[2]);
                    long s0 = IDX(o, i + sh[0], j + sh[1], k + sh[2]);
                    double pl = P[s1], pr = P[ib];
                    if (!first) {
                        pl = P[s1] + 0.5 * limit(o->limiter, P[s1] - P[s2], P[ib] - P[s1]);
                        pr = P[ib] - 0.5 * limit(o->limiter, P[ib] - P[s1], P[s0] - P[ib]);
                    }
                    double ch = o->glm_ch, bl = wl[B1 + d], brr = wr[B1 + d];
                    double bs = 0.5 * (bl + brr) - 0.5 * (pr - pl) / ch;
                    double ps = 0.5 * (pl + pr) - 0.5 * ch * (brr - bl);
                    f[B1 + d] = ps;
                    o->FP[d][ib] = ch * ch * bs;
                }
                store(o, o->F[d], IDX(o, i, j, k), f);
            }
}

/* div B at cell (i,j,k): (1/V) sum_d [A+ (B_d(c) + B_d(c+e_d))/2 - A- (B_d(c-e_d) + B_d(c))/2] */
static double divb_cell(const orc_t *o, const double *U, int i, int j, int k)
{
    int c3[3] = {i, j, k};
    double s = 0.0;
    for (int d = 0; d < 3; d++) {
        int pl[3] = {i, j, k}, mi[3] = {i, j, k};
        pl[d] += 1; mi[d] -= 1;
        double bc = U[(B1 + d) * o->nt + IDX(o, c3[0], c3[1], c3[2])];
        double bp = U[(B1 + d) * o->nt + IDX(o, pl[0], pl[1], pl[2])];
        double bm = U[(B1 + d) * o->nt + IDX(o, mi[0], mi[1], mi[2])];
        s += area(o, d, pl[0], pl[1], pl[2]) * 0.5 * (bc + bp) - area(o, d, i, j, k) * 0.5 * (bm + bc);
    }
    return s / volume(o, i, j, k);
}

static void residual(orc_t *o, const double *U, double dt)
{
    all_prims(o, U);
    for (int d = 0; d < 3; d++) face_fluxes(o, d);
    if (o->divb == DIVB_LINDE) {
#pragma omp parallel for collapse(2)
        for (int k = -1; k <= o->n[2]; k++)
            for (int j = -1; j <= o->n[1]; j++)
                for (int i = -1; i <= o->n[0]; i++) o->divB[IDX(o, i, j, k)] = divb_cell(o, U, i, j, k);
    }
    double Om = o->omega;
#pragma omp parallel for collapse(2)
    for (int k = 0; k < o->n[2]; k++)
        for (int j = 0; j < o->n[1]; j++)
            for (int i = 0; i < o->n[0]; i++) {
                long id = IDX(o, i, j, k);
                double V = volume(o, i, j, k);
                double Lc[NV], w[NV];
                int sh[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
                for (int v = 0; v < NV; v++) Lc[v] = 0.0;
                if (o->divb == DIVB_GLM) o->LPsi[id] = 0.0;
                /* flux divergence: -(1/V) sum_d (A+ F+ - A- F-) */
                for (int d = 0; d < 3; d++) {
                    long idp = IDX(o, i + sh[d][0], j + sh[d][1], k + sh[d][2]);
                    double am = area(o, d, i, j, k);
                    double ap = area(o, d, i + sh[d][0], j + sh[d][1], k + sh[d][2]);
                    for (int v = 0; v < NV; v++)
                        Lc[v] -= (ap * o->F[d][v * o->nt + idp] - am * o->F[d][v * o->nt + id]) / V;
                    if (o->divb == DIVB_GLM) {
                        /* the flux form of grad psi leaves psi (A+ - A-) / V, as for p_tot */
                        Lc[B1 + d] += o->Pcur[id] * (ap - am) / V;
                        o->LPsi[id] -= (ap * o->FP[d][idp] - am * o->FP[d][id]) / V;
                    }
                }
                load(o, o->W, id, w);
                double rho = w[0], vr = w[1], vt = w[2], vp = w[3];
                double br = w[5], bt = w[6], bp = w[7];
                if (o->geom == GEOM_SPH) {
                    double r = ctr(o, 0, i), th = ctr(o, 1, j), ph = ctr(o, 2, k);
                    double cot = cos(th) / sin(th);
                    double ptot = w[4] + 0.5 * (br * br + bt * bt + bp * bp);
                    /* geometric terms of div(rho v v + p_tot I - B B) and div(v B - B v) in
                     * spherical components; the p_tot parts use face-area differences */
                    double dAr = area(o, 0, i + 1, j, k) - area(o, 0, i, j, k);
                    double dAt = area(o, 1, i, j + 1, k) - area(o, 1, i, j, k);
                    Lc[M1] += ptot * dAr / V + (rho * (vt * vt + vp * vp) - (bt * bt + bp * bp)) / r;
                    Lc[M2] += ptot * dAt / V + (-(rho * vr * vt - br * bt) + cot * (rho * vp * vp - bp * bp)) / r;
                    Lc[M3] += -((rho * vp * vr - bp * br) + cot * (rho * vp * vt - bp * bt)) / r;
                    Lc[B2] += (vr * bt - vt * br) / r;
                    Lc[B3] += ((vr * bp - vp * br) + cot * (vt * bp - vp * bt)) / r;
                    if (Om != 0.0) {
                        /* F = rho (Omega x r) x Omega + 2 rho v x Omega, Omega = Omega z-hat,
                         * evaluated with Cartesian cross products, then projected */
                        double er[3] = {sin(th) * cos(ph), sin(th) * sin(ph), cos(th)};
                        double et[3] = {cos(th) * cos(ph), cos(th) * sin(ph), -sin(th)};
                        double ep[3] = {-sin(ph), cos(ph), 0.0};
                        double Ov[3] = {0.0, 0.0, Om};
                        double rv[3], vv[3], t1[3], cen[3], cor[3], F[3];
                        for (int c = 0; c < 3; c++) {
                            rv[c] = r * er[c];
                            vv[c] = vr * er[c] + vt * et[c] + vp * ep[c];
                        }
                        t1[0] = Ov[1] * rv[2] - Ov[2] * rv[1];          /* Omega x r */
                        t1[1] = Ov[2] * rv[0] - Ov[0] * rv[2];
                        t1[2] = Ov[0] * rv[1] - Ov[1] * rv[0];
                        cen[0] = t1[1] * Ov[2] - t1[2] * Ov[1];         /* (Omega x r) x Omega */
                        cen[1] = t1[2] * Ov[0] - t1[0] * Ov[2];
                        cen[2] = t1[0] * Ov[1] - t1[1] * Ov[0];
                        cor[0] = vv[1] * Ov[2] - vv[2] * Ov[1];         /* v x Omega */
                        cor[1] = vv[2] * Ov[0] - vv[0] * Ov[2];
                        cor[2] = vv[0] * Ov[1] - vv[1] * Ov[0];
                        for (int c = 0; c < 3; c++) F[c] = rho * cen[c] + 2.0 * rho * cor[c];
                        Lc[M1] += F[0] * er[0] + F[1] * er[1] + F[2] * er[2];
                        Lc[M2] += F[0] * et[0] + F[1] * et[1] + F[2] * et[2];
                        Lc[M3] += F[0] * ep[0] + F[1] * ep[1] + F[2] * ep[2];
                        Lc[EN] += vv[0] * F[0] + vv[1] * F[1] + vv[2] * F[2];
                    }
                    if (o->gravity) {
                        /* the paper writes g = GM/r^2 e_r; read as the inward pull -GM/r^2 e_r */
                        double g = o->gm / (r * r);
                        Lc[M1] -= rho * g;
                        Lc[EN] -= rho * vr * g;
                    }
                }
                if (o->divb == DIVB_LINDE) {
                    /* Linde-type diffusion: dB/dt += grad(eta div B), de/dt += B . grad(eta div B),
                     * eta = C_d / (dt sum_d 1/dx_d^2), central differences of cell-centred div B */
                    double sinv = 0.0, gr[3];
                    for (int d = 0; d < 3; d++) {
                        double wd = width(o, d, i, j, k);
                        sinv += 1.0 / (wd * wd);
                    }
                    double eta = o->divb_coef / (dt * sinv);
                    for (int d = 0; d < 3; d++) {
                        int pl[3] = {i, j, k}, mi[3] = {i, j, k};
                        pl[d] += 1; mi[d] -= 1;
                        double dd = o->divB[IDX(o, pl[0], pl[1], pl[2])] - o->divB[IDX(o, mi[0], mi[1], mi[2])];
                        double dx = ctr(o, d, pl[d]) - ctr(o, d, mi[d]);
                        if (o->geom == GEOM_SPH && d == 1) dx = ctr(o, 0, i) * dx;
                        if (o->geom == GEOM_SPH && d == 2) dx = ctr(o, 0, i) * sin(ctr(o, 1, j)) * dx;
                        gr[d] = eta * dd / dx;
                    }
                    Lc[B1] += gr[0]; Lc[B2] += gr[1]; Lc[B3] += gr[2];
                    Lc[EN] += br * gr[0] + bt * gr[1] + bp * gr[2];
                }
                if (o->divb == DIVB_POWELL) {
                    /* Powell's eight-wave source -(div B) (0, B, v.B, v), the cell's own div B */
                    double db = divb_cell(o, U, i, j, k);
                    Lc[M1] -= db * br; Lc[M2] -= db * bt; Lc[M3] -= db * bp;
                    Lc[EN] -= db * (vr * br + vt * bt + vp * bp);
                    Lc[B1] -= db * vr; Lc[B2] -= db * vt; Lc[B3] -= db * vp;
                }
                store(o, o->L, id, Lc);
            }
}

/* ---- floors and CFL ------------------------------------------------------------------------ */
static void apply_floors(orc_t *o, double *U)
{
    long hits = 0;
    int bad = 0;
#pragma omp parallel for collapse(2) reduction(+ : hits) reduction(| : bad)
    for (int k = 0; k < o->n[2]; k++)
        for (int j = 0; j < o->n[1]; j++)
            for (int i = 0; i < o->n[0]; i++) {
                long id = IDX(o, i, j, k);
                double u[NV], w[NV];
                load(o, U, id, u);
                for (int v = 0; v < NV; v++) if (!isfinite(u[v])) bad = 1;
                if (u[RHO] < o->rho_floor) { u[RHO] = o->rho_floor; hits++; }
                cons2prim(o, u, w);
                if (w[4] < o->p_floor) {
                    w[4] = o->p_floor;
                    prim2cons(o, w, u);
                    hits++;
                }
                store(o, U, id, u);
            }
    o->floor_hits += hits;
    if (bad) o->status = 1;
}

/* dt = CFL / max_cells sum_d (|v_d| + c_f,d) / dx_d over interior cells */
static double cfl_dt(orc_t *o, const double *U)
{
    double smax = 0.0;
#pragma omp parallel for collapse(2) reduction(max : smax)
    for (int k = 0; k < o->n[2]; k++)
        for (int j = 0; j < o->n[1]; j++)
            for (int i = 0; i < o->n[0]; i++) {
                double u[NV], w[NV], s = 0.0;
                load(o, U, IDX(o, i, j, k), u);
                cons2prim(o, u, w);
                for (int d = 0; d < 3; d++) s += (fabs(w[1 + d]) + fast_speed(o, w, d)) / width(o, d, i, j, k);
                if (s > smax) smax = s;
            }
    return o->cfl / smax;
}

/* ---- public API ---------------------------------------------------------------------------- */
void orc_destroy(orc_t *o);

orc_t *orc_create(const int *ig, const double *dg, double gamma, double omega_si, const double *od, const int *oi)
{
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    for (int d = 0; d < 3; d++) { o->n[d] = ig[d]; o->xmin[d] = dg[2 * d]; o->xmax[d] = dg[2 * d + 1]; }
    o->geom = ig[3]; o->stretch = ig[4];
    for (int s = 0; s < 6; s++) o->bc[s] = ig[5 + s];
    o->band_refine = ig[11]; o->band_lo = dg[6]; o->band_hi = dg[7];
    for (int d = 0; d < 3; d++) o->p[d] = o->n[d] + 2 * NG;
    o->nt = (long)o->p[0] * o->p[1] * o->p[2];
    for (int d = 0; d < 3; d++) {
        o->e[d] = (double *)malloc(sizeof(double) * (o->n[d] + 2 * NG + 1));
        o->c[d] = (double *)malloc(sizeof(double) * (o->n[d] + 2 * NG));
        for (int i = -NG; i <= o->n[d] + NG; i++) o->e[d][i + NG] = edge_pos(o, d, i);
        for (int i = -NG; i < o->n[d] + NG; i++) o->c[d][i + NG] = 0.5 * (o->e[d][i + NG] + o->e[d][i + NG + 1]);
    }
    o->t0 = O_AU / O_V0;
    double rho0 = O_MP * O_N0;
    o->p0 = rho0 * O_V0 * O_V0;
    o->b0 = sqrt(O_MU0 * rho0) * O_V0;
    o->gamma = gamma;
    o->omega_si = omega_si;
    o->omega = omega_si * o->t0;
    o->cfl = od[0]; o->divb_coef = od[1]; o->rho_floor = od[2]; o->p_floor = od[3];
    o->glm_alpha = od[4];
    o->limiter = oi[0]; o->flux = oi[1]; o->gravity = oi[2]; o->divb = oi[3]; o->init_vphi = oi[4];
    o->cme_model = oi[5];
    o->tracer = oi[6];
    o->gm = O_GM / (O_AU * O_V0 * O_V0);
    if (o->geom == GEOM_CART) { o->omega = 0.0; o->gravity = 0; }
    size_t sz = sizeof(double) * NV * o->nt;
    o->U = (double *)calloc(1, sz); o->U0 = (double *)calloc(1, sz); o->U1 = (double *)calloc(1, sz);
    o->L = (double *)calloc(1, sz); o->W = (double *)calloc(1, sz); o->Ufix = (double *)calloc(1, sz);
    for (int d = 0; d < 3; d++) o->F[d] = (double *)calloc(1, sz);
    o->divB = (double *)calloc(1, sizeof(double) * o->nt);
    o->T = (double *)calloc(1, sizeof(double) * o->nt); o->T0 = (double *)calloc(1, sizeof(double) * o->nt);
    o->T1 = (double *)calloc(1, sizeof(double) * o->nt); o->LT = (double *)calloc(1, sizeof(double) * o->nt);
    o->C = (double *)calloc(1, sizeof(double) * o->nt);
    o->Psi = (double *)calloc(1, sizeof(double) * o->nt); o->Psi0 = (double *)calloc(1, sizeof(double) * o->nt);
    o->Psi1 = (double *)calloc(1, sizeof(double) * o->nt); o->LPsi = (double *)calloc(1, sizeof(double) * o->nt);
    for (int d = 0; d < 3; d++) o->FP[d] = (double *)calloc(1, sizeof(double) * o->nt);
    o->Pcur = o->Psi;
    /* smallest cell width over the interior (dr, r dtheta, r sin(theta) dphi on the sphere) */
    o->glm_dmin = 1e300;
    for (int k = 0; k < o->n[2]; k++)
        for (int j = 0; j < o->n[1]; j++)
            for (int i = 0; i < o->n[0]; i++)
                for (int d = 0; d < 3; d++) o->glm_dmin = fmin(o->glm_dmin, width(o, d, i, j, k));
    return o;
}

void orc_destroy(orc_t *o)
{
    if (!o) return;
    for (int d = 0; d < 3; d++) { free(o->e[d]); free(o->c[d]); free(o->F[d]); }
    free(o->U); free(o->U0); free(o->U1); free(o->L); free(o->W); free(o->Ufix); free(o->divB);
    free(o->T); free(o->T0); free(o->T1); free(o->LT); free(o->C);
    free(o->Psi); free(o->Psi0); free(o->Psi1); free(o->LPsi);
    for (int d = 0; d < 3; d++) free(o->FP[d]);
    free(o->tm); free(o->maps); free(o->cme);
    free(o);
}

/* maps in SI [n_maps][5][n2][n3] (v_r, n, p, B_r, B_phi), times in s; CMEs in SI [n_cme][8] */
int orc_set_boundary(orc_t *o, int n_maps, const double *t_si, const double *maps_si, int n_cme, const double *cme_si)
{
    free(o->tm); free(o->maps); free(o->cme);
    long per = 5L * o->n[1] * o->n[2];
    o->n_maps = n_maps;
    o->tm = (double *)malloc(sizeof(double) * (n_maps > 0 ? n_maps : 1));
    o->maps = (double *)malloc(sizeof(double) * per * (n_maps > 0 ? n_maps : 1));
    for (int m = 0; m < n_maps; m++) {
        o->tm[m] = t_si[m] / o->t0;
        for (long q = 0; q < per / 5; q++) {
            const double *src = maps_si + (long)m * per;
            double *dst = o->maps + (long)m * per;
            dst[0 * (per / 5) + q] = src[0 * (per / 5) + q] / O_V0;
            dst[1 * (per / 5) + q] = src[1 * (per / 5) + q] / O_N0;
            dst[2 * (per / 5) + q] = src[2 * (per / 5) + q] / o->p0;
            dst[3 * (per / 5) + q] = src[3 * (per / 5) + q] / o->b0;
            dst[4 * (per / 5) + q] = src[4 * (per / 5) + q] / o->b0;
        }
    }
    o->n_cme = n_cme;
    o->cme = (double *)malloc(sizeof(double) * 8 * (n_cme > 0 ? n_cme : 1));
    for (int c = 0; c < n_cme; c++) {
        const double *s = cme_si + 8 * c;
        double *d = o->cme + 8 * c;
        d[0] = s[0] / o->t0; d[1] = s[1] / o->t0; d[2] = s[2]; d[3] = s[3]; d[4] = s[4];
        d[5] = s[5] / O_V0;
        d[6] = s[6] / O_N0;
        d[7] = 2.0 * s[6] * O_KB * s[7] / o->p0;    /* p = 2 n k_B T */
    }
    return 0;
}

/* initial state (Sect. 2.1): the boundary map at the current time, extended radially by the
 * expansion laws v_r const, n ~ r^-2, p ~ r^-2gamma, B_r ~ r^-2, with the spiral B_phi = -B_r Omega
 * r sin(theta) / v_r and v_theta = B_theta = 0. v_phi (the paper names no value): 0 in the
 * co-rotating frame (init_vphi = 0), or the inertially radial flow seen from the rotating frame,
 * v_phi = -Omega r sin(theta), parallel to the spiral field (init_vphi = 1) */
int orc_init_state(orc_t *o)
{
    if (o->geom != GEOM_SPH || o->n_maps < 1) return -1;
    double rin = o->xmin[0];
    for (int k = 0; k < o->n[2]; k++)
        for (int j = 0; j < o->n[1]; j++) {
            double b[5];
            map_value(o, o->t, j, k, b);
            for (int i = 0; i < o->n[0]; i++) {
                double r = ctr(o, 0, i), th = ctr(o, 1, j);
                double x = rin / r;
                double w[NV], u[NV];
                w[0] = b[1] * x * x;
                w[1] = b[0]; w[2] = 0.0;
                w[3] = o->init_vphi ? -o->omega * r * sin(th) : 0.0;
                w[4] = b[2] * pow(x, 2.0 * o->gamma);
                w[5] = b[3] * x * x; w[6] = 0.0;
                w[7] = -w[5] * o->omega * r * sin(th) / w[1];
                prim2cons(o, w, u);
                store(o, o->U, IDX(o, i, j, k), u);
            }
        }
    return 0;
}

/* interior state [8][n3][n2][n1], r fastest, code units */
void orc_set_state(orc_t *o, const double *Uin, double t)
{
    for (int v = 0; v < NV; v++)
        for (int k = 0; k < o->n[2]; k++)
            for (int j = 0; j < o->n[1]; j++)
                for (int i = 0; i < o->n[0]; i++)
                    o->U[v * o->nt + IDX(o, i, j, k)] = Uin[(((long)v * o->n[2] + k) * o->n[1] + j) * o->n[0] + i];
    o->t = t;
}

void orc_get_state(const orc_t *o, double *Uout, double *t)
{
    for (int v = 0; v < NV; v++)
        for (int k = 0; k < o->n[2]; k++)
            for (int j = 0; j < o->n[1]; j++)
                for (int i = 0; i < o->n[0]; i++)
                    Uout[(((long)v * o->n[2] + k) * o->n[1] + j) * o->n[0] + i] = o->U[v * o->nt + IDX(o, i, j, k)];
    if (t) *t = o->t;
}

/* padded state [8][p3][p2][p1] including ghosts; for BC_FIXED faces the ghost values given here
 * are kept for the whole run */
void orc_set_state_padded(orc_t *o, const double *Up, double t)
{
    memcpy(o->U, Up, sizeof(double) * NV * o->nt);
    memcpy(o->Ufix, Up, sizeof(double) * NV * o->nt);
    o->t = t;
}

void orc_get_state_padded(const orc_t *o, double *Up) { memcpy(Up, o->U, sizeof(double) * NV * o->nt); }

void orc_fill_ghosts(orc_t *o, double tau) { fill_ghosts(o, o->U, tau); }

double orc_cfl_dt(orc_t *o) { return cfl_dt(o, o->U); }

/* the floors of one stage end applied to the interior state (test access; counts into floor_hits) */
void orc_apply_floors(orc_t *o) { apply_floors(o, o->U); }

/* the n + 1 interior edges of direction d */
void orc_edges(const orc_t *o, int d, double *out)
{
    for (int i = 0; i <= o->n[d]; i++) out[i] = o->e[d][i + NG];
}

/* one SSP-RK2 step: U1 = U + dt L(U, t); U <- U/2 + (U1 + dt L(U1, t + dt))/2; floors after each
 * stage; dt = CFL bound, capped by dt_max when dt_max > 0. Returns dt, or -1 on non-finite state */
/* ---- GLM psi: ghost layers copied like the other variables (zero gradient at the driven face),
 * each direction over the ghost layers of the previous ones, as the MHD ghost fill does */
static void psi_fill(orc_t *o, double *P)
{
    for (int d = 0; d < 3; d++)
        for (int side = 0; side < 2; side++) {
            int bc = o->bc[2 * d + side], n = o->n[d];
            int a_lo = -NG, a_hi = o->n[(d + 1) % 3] + NG, b_lo = -NG, b_hi = o->n[(d + 2) % 3] + NG;
            if (d == 0) { a_lo = 0; a_hi = o->n[1]; b_lo = 0; b_hi = o->n[2]; }
            if (d == 1) { a_lo = 0; a_hi = o->n[2]; b_lo = -NG; b_hi = o->n[0] + NG; }
            for (int b = b_lo; b < b_hi; b++)
                for (int a = a_lo; a < a_hi; a++)
                    for (int g = 1; g <= NG; g++) {
                        int gi = side == 0 ? -g : n - 1 + g, src;
                        if (bc == BC_CONT || bc == BC_DRIVEN) src = side == 0 ? 0 : n - 1;
                        else if (bc == BC_REFLECT) src = side == 0 ? g - 1 : n - g;
                        else if (bc == BC_PERIODIC) src = ((gi % n) + n) % n;
                        else src = gi;   /* FIXED: keep */
                        P[cell_id(o, d, gi, a, b)] = P[cell_id(o, d, src, a, b)];
                    }
        }
}

/* ---- CME tracer (a passive scalar c carried by the plasma; rho c is conserved) --------------
 * The paper marks inserted CME plasma with a tracer. Boundary: c = 1 in the ghost columns inside
 * the CME footprint while it is inserted, 0 elsewhere on the driven face; c is copied like the
 * other variables on every other face. Face flux: F_rho times the limited linear reconstruction
 * of c on the upwind side of the mass flux (the same limiter as the MHD variables), so that c = 1
 * everywhere moves rho c exactly like rho. After each stage rho c is clipped to [0, rho]. */
static void tracer_fill_side(orc_t *o, double *T, const double *U, int d, int side, double tau)
{
    int bc = o->bc[2 * d + side];
    int n = o->n[d];
    int a_lo = -NG, a_hi = o->n[(d + 1) % 3] + NG, b_lo = -NG, b_hi = o->n[(d + 2) % 3] + NG;
    if (d == 0) { a_lo = 0; a_hi = o->n[1]; b_lo = 0; b_hi = o->n[2]; }
    if (d == 1) { a_lo = 0; a_hi = o->n[2]; b_lo = -NG; b_hi = o->n[0] + NG; }
    if (bc == BC_DRIVEN) {
        for (int k = 0; k < o->n[2]; k++)
            for (int j = 0; j < o->n[1]; j++) {
                double q[5] = {0, 0, 0, 0, 0};
                int hit = cme_hit(o, tau, j, k, q);
                for (int g = 1; g <= NG; g++) {
                    long id = IDX(o, -g, j, k);
                    T[id] = hit ? U[RHO * o->nt + id] : 0.0;
                }
            }
        return;
    }
    for (int b = b_lo; b < b_hi; b++)
        for (int a = a_lo; a < a_hi; a++)
            for (int g = 1; g <= NG; g++) {
                int gi = side == 0 ? -g : n - 1 + g;
                int src;
                if (bc == BC_CONT) src = side == 0 ? 0 : n - 1;
                else if (bc == BC_REFLECT) src = side == 0 ? g - 1 : n - g;
                else if (bc == BC_PERIODIC) src = ((gi % n) + n) % n;
                else src = gi;   /* FIXED: keep */
                T[cell_id(o, d, gi, a, b)] = T[cell_id(o, d, src, a, b)];
            }
}

static void tracer_fill(orc_t *o, double *T, const double *U, double tau)
{
    for (int d = 0; d < 3; d++)
        for (int side = 0; side < 2; side++) tracer_fill_side(o, T, U, d, side, tau);
}

/* residual of rho c, with the mass fluxes of the residual just evaluated for U (o->F) */
static void tracer_residual(orc_t *o, const double *T, const double *U)
{
#pragma omp parallel for
    for (long id = 0; id < o->nt; id++) {
        double rho = U[RHO * o->nt + id];
        o->C[id] = rho != 0.0 ? T[id] / rho : 0.0;
    }
    const int sh[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma omp parallel for collapse(2)
    for (int k = 0; k < o->n[2]; k++)
        for (int j = 0; j < o->n[1]; j++)
            for (int i = 0; i < o->n[0]; i++) {
                long id = IDX(o, i, j, k);
                double V = volume(o, i, j, k), l = 0.0;
                for (int d = 0; d < 3; d++) {
                    double ft[2];
                    for (int s = 0; s < 2; s++) {      /* lower (s = 0) and upper face along d */
                        int b[3] = {i + s * sh[d][0], j + s * sh[d][1], k + s * sh[d][2]};
                        long ib = IDX(o, b[0], b[1], b[2]);
                        long st = d == 0 ? 1 : (d == 1 ? o->p[0] : (long)o->p[0] * o->p[1]);
                        double cm2 = o->C[ib - 2 * st], cm1 = o->C[ib - st], c0 = o->C[ib], cp1 = o->C[ib + st];
                        double cl = cm1 + 0.5 * limit(o->limiter, cm1 - cm2, c0 - cm1);
                        double cr = c0 - 0.5 * limit(o->limiter, c0 - cm1, cp1 - c0);
                        double fr = o->F[d][RHO * o->nt + ib];
                        ft[s] = fr * (fr >= 0.0 ? cl : cr);
                    }
                    double am = area(o, d, i, j, k);
                    double ap = area(o, d, i + sh[d][0], j + sh[d][1], k + sh[d][2]);
                    l -= (ap * ft[1] - am * ft[0]) / V;
                }
                o->LT[id] = l;
            }
}

static void tracer_clip(orc_t *o, double *T, const double *U)
{
    for (int k = 0; k < o->n[2]; k++)
        for (int j = 0; j < o->n[1]; j++)
            for (int i = 0; i < o->n[0]; i++) {
                long id = IDX(o, i, j, k);
                double rho = U[RHO * o->nt + id];
                T[id] = fmin(fmax(T[id], 0.0), rho);
            }
}

double orc_step(orc_t *o, double dt_max)
{
    double dt = cfl_dt(o, o->U);
    if (dt_max > 0.0 && dt > dt_max) dt = dt_max;
    long tot = NV * o->nt;
    const int glm = o->divb == DIVB_GLM;
    if (glm) {
        /* c_h: the fastest speed the step's dt carries at the CFL number over the smallest cell */
        o->glm_ch = o->cfl * o->glm_dmin / dt;
        memcpy(o->Psi0, o->Psi, sizeof(double) * o->nt);
        psi_fill(o, o->Psi);
        o->Pcur = o->Psi;
    }
    memcpy(o->U0, o->U, sizeof(double) * tot);
    fill_ghosts(o, o->U, o->t);
    residual(o, o->U, dt);
    if (o->tracer) {
        memcpy(o->T0, o->T, sizeof(double) * o->nt);
        tracer_fill(o, o->T, o->U, o->t);
        tracer_residual(o, o->T, o->U);
        memcpy(o->T1, o->T, sizeof(double) * o->nt);
        for (int k = 0; k < o->n[2]; k++)
            for (int j = 0; j < o->n[1]; j++)
                for (int i = 0; i < o->n[0]; i++) {
                    long id = IDX(o, i, j, k);
                    o->T1[id] = o->T0[id] + dt * o->LT[id];
                }
    }
    memcpy(o->U1, o->U, sizeof(double) * tot);
    for (int v = 0; v < NV; v++)
        for (int k = 0; k < o->n[2]; k++)
            for (int j = 0; j < o->n[1]; j++)
                for (int i = 0; i < o->n[0]; i++) {
                    long id = v * o->nt + IDX(o, i, j, k);
                    o->U1[id] = o->U0[id] + dt * o->L[id];
                }
    apply_floors(o, o->U1);
    if (o->tracer) tracer_clip(o, o->T1, o->U1);
    if (glm) {
        for (int k = 0; k < o->n[2]; k++)
            for (int j = 0; j < o->n[1]; j++)
                for (int i = 0; i < o->n[0]; i++) {
                    long id = IDX(o, i, j, k);
                    o->Psi1[id] = o->Psi0[id] + dt * o->LPsi[id];
                }
        psi_fill(o, o->Psi1);
        o->Pcur = o->Psi1;
    }
    fill_ghosts(o, o->U1, o->t + dt);
    residual(o, o->U1, dt);
    if (o->tracer) {
        tracer_fill(o, o->T1, o->U1, o->t + dt);
        tracer_residual(o, o->T1, o->U1);
        for (int k = 0; k < o->n[2]; k++)
            for (int j = 0; j < o->n[1]; j++)
                for (int i = 0; i < o->n[0]; i++) {
                    long id = IDX(o, i, j, k);
                    o->T[id] = 0.5 * o->T0[id] + 0.5 * (o->T1[id] + dt * o->LT[id]);
                }
    }
    for (int v = 0; v < NV; v++)
        for (int k = 0; k < o->n[2]; k++)
            for (int j = 0; j < o->n[1]; j++)
                for (int i = 0; i < o->n[0]; i++) {
                    long id = v * o->nt + IDX(o, i, j, k);
                    o->U[id] = 0.5 * o->U0[id] + 0.5 * (o->U1[id] + dt * o->L[id]);
                }
    apply_floors(o, o->U);
    if (o->tracer) tracer_clip(o, o->T, o->U);
    if (glm) {
        /* second stage, then the damping source -(c_h^2 / c_p^2) psi integrated exactly over the
         * step (operator split): psi *= exp(-alpha c_h dt / dmin) */
        const double damp = exp(-o->glm_alpha * o->glm_ch * dt / o->glm_dmin);
        for (int k = 0; k < o->n[2]; k++)
            for (int j = 0; j < o->n[1]; j++)
                for (int i = 0; i < o->n[0]; i++) {
                    long id = IDX(o, i, j, k);
                    o->Psi[id] = (0.5 * o->Psi0[id] + 0.5 * (o->Psi1[id] + dt * o->LPsi[id])) * damp;
                }
    }
    o->t = o->t + dt;
    return o->status ? -1.0 : dt;
}

/* tracer values c of the interior cells, [n3][n2][n1]: set (rho c from the current rho) / get */
void orc_set_tracer(orc_t *o, const double *c)
{
    for (int k = 0; k < o->n[2]; k++)
        for (int j = 0; j < o->n[1]; j++)
            for (int i = 0; i < o->n[0]; i++) {
                long id = IDX(o, i, j, k);
                o->T[id] = o->U[RHO * o->nt + id] * c[((long)k * o->n[1] + j) * o->n[0] + i];
            }
}

void orc_get_tracer(const orc_t *o, double *c)
{
    for (int k = 0; k < o->n[2]; k++)
        for (int j = 0; j < o->n[1]; j++)
            for (int i = 0; i < o->n[0]; i++) {
                long id = IDX(o, i, j, k);
                c[((long)k * o->n[1] + j) * o->n[0] + i] = o->T[id] / o->U[RHO * o->nt + id];
            }
}

/* GLM psi of the interior cells [n3][n2][n1]: set / get; c_h of the last step */
void orc_set_psi(orc_t *o, const double *p)
{
    for (int k = 0; k < o->n[2]; k++)
        for (int j = 0; j < o->n[1]; j++)
            for (int i = 0; i < o->n[0]; i++) o->Psi[IDX(o, i, j, k)] = p[((long)k * o->n[1] + j) * o->n[0] + i];
}

void orc_get_psi(const orc_t *o, double *p)
{
    for (int k = 0; k < o->n[2]; k++)
        for (int j = 0; j < o->n[1]; j++)
            for (int i = 0; i < o->n[0]; i++) p[((long)k * o->n[1] + j) * o->n[0] + i] = o->Psi[IDX(o, i, j, k)];
}

double orc_glm_ch(const orc_t *o) { return o->glm_ch; }
double orc_glm_dmin(const orc_t *o) { return o->glm_dmin; }

/* residual L(U) at the current state and time (ghosts filled at tau), interior [8][n3][n2][n1] */
void orc_residual(orc_t *o, double tau, double dt, double *Lout)
{
    fill_ghosts(o, o->U, tau);
    residual(o, o->U, dt);
    for (int v = 0; v < NV; v++)
        for (int k = 0; k < o->n[2]; k++)
            for (int j = 0; j < o->n[1]; j++)
                for (int i = 0; i < o->n[0]; i++)
                    Lout[(((long)v * o->n[2] + k) * o->n[1] + j) * o->n[0] + i] = o->L[v * o->nt + IDX(o, i, j, k)];
}

/* div B of the current state (ghosts as they are) at interior cells [n3][n2][n1] */
void orc_divb(orc_t *o, double *out)
{
    for (int k = 0; k < o->n[2]; k++)
        for (int j = 0; j < o->n[1]; j++)
            for (int i = 0; i < o->n[0]; i++)
                out[((long)k * o->n[1] + j) * o->n[0] + i] = divb_cell(o, o->U, i, j, k);
}

/* cell volumes [n3][n2][n1] (for conservation sums) */
void orc_volumes(const orc_t *o, double *out)
{
    for (int k = 0; k < o->n[2]; k++)
        for (int j = 0; j < o->n[1]; j++)
            for (int i = 0; i < o->n[0]; i++) out[((long)k * o->n[1] + j) * o->n[0] + i] = volume(o, i, j, k);
}

/* centres of direction d, [n_d + 4] including ghosts */
void orc_centres(const orc_t *o, int d, double *out) { memcpy(out, o->c[d], sizeof(double) * (o->n[d] + 2 * NG)); }

/* boundary column values at time tau (map interpolation + CME), [5][n2][n3] code units
 * (rho, v_r, p, B_r, B_phi); also the CME hit mask [n2][n3] */
void orc_boundary_values(orc_t *o, double tau, double *out, int *hit)
{
    long per = (long)o->n[1] * o->n[2];
    for (int j = 0; j < o->n[1]; j++)
        for (int k = 0; k < o->n[2]; k++) {
            double b[5];
            map_value(o, tau, j, k, b);
            double q[5] = {b[1], b[0], b[2], b[3], b[4]};
            int h = cme_hit(o, tau, j, k, q);
            for (int f = 0; f < 5; f++) out[f * per + (long)j * o->n[2] + k] = q[f];
            if (hit) hit[(long)j * o->n[2] + k] = h;
        }
}

long orc_floor_hits(const orc_t *o) { return o->floor_hits; }
double orc_time(const orc_t *o) { return o->t; }
void orc_scales(const orc_t *o, double *s)
{
    s[0] = o->t0; s[1] = o->p0; s[2] = o->b0; s[3] = o->omega; s[4] = o->gm;
}

/* ---- probe sampling (Sect. 2: massless sampling points moving along trajectories) ---------- */
/* knots [n_probes][n_knots][4] = (t s, r m, lat rad, lon_inertial rad). At the current time:
 * linear interpolation between the bracketing knots (clamped), co-rotating longitude
 * phi = lon - Omega t wrapped to [0, 2 pi), theta = pi/2 - lat; the 2x2x2 cell centres around
 * the point (found by scanning the centre arrays), trilinear weights, primitives interpolated.
 * out [n_probes][13] = (t s, n m^-3, v_r, v_theta, v_phi (inertial) m/s, B_r, B_theta, B_phi T,
 *                       p Pa, |B| T, i, j, k) */
void orc_sample(const orc_t *o, int n_probes, int n_knots, const double *traj, double *out)
{
    double tsi = o->t * o->t0;
    const double twopi = 2.0 * O_PI;
    for (int p = 0; p < n_probes; p++) {
        const double *kn = traj + (long)p * n_knots * 4;
        int a = 0;
        double w = 0.0;
        if (n_knots == 1 || tsi <= kn[0]) { a = 0; w = 0.0; }
        else if (tsi >= kn[(n_knots - 1) * 4]) { a = n_knots - 2; w = 1.0; }
        else {
            while (a + 1 < n_knots - 1 && kn[(a + 1) * 4] <= tsi) a++;
            w = (tsi - kn[a * 4]) / (kn[(a + 1) * 4] - kn[a * 4]);
        }
        int b = (n_knots == 1) ? 0 : a + 1;
        double rm = kn[a * 4 + 1] + w * (kn[b * 4 + 1] - kn[a * 4 + 1]);
        double lat = kn[a * 4 + 2] + w * (kn[b * 4 + 2] - kn[a * 4 + 2]);
        double lon = kn[a * 4 + 3] + w * (kn[b * 4 + 3] - kn[a * 4 + 3]);
        double r = rm / O_AU;
        double th = O_PI / 2.0 - lat;
        double ph = lon - o->omega_si * tsi;
        ph = ph - twopi * floor(ph / twopi);
        if (ph >= twopi) ph = 0.0;
        /* r, theta: largest centre index in [0, n-2] not above the position (0 if none) */
        int i = 0, j = 0, k;
        for (int q = 0; q <= o->n[0] - 2; q++) if (ctr(o, 0, q) <= r) i = q;
        for (int q = 0; q <= o->n[1] - 2; q++) if (ctr(o, 1, q) <= th) j = q;
        double wr = o->n[0] > 1 ? (r - ctr(o, 0, i)) / (ctr(o, 0, i + 1) - ctr(o, 0, i)) : 0.0;
        double wt = o->n[1] > 1 ? (th - ctr(o, 1, j)) / (ctr(o, 1, j + 1) - ctr(o, 1, j)) : 0.0;
        wr = fmin(fmax(wr, 0.0), 1.0);
        wt = fmin(fmax(wt, 0.0), 1.0);
        /* phi: periodic; below the first centre the bracket is (n3-1, 0) across 2 pi */
        k = o->n[2] - 1;
        double phk = ctr(o, 2, o->n[2] - 1) - twopi;
        for (int q = 0; q < o->n[2]; q++) if (ctr(o, 2, q) <= ph) { k = q; phk = ctr(o, 2, q); }
        double dph = hi(o, 2, 0) - lo(o, 2, 0);
        double wp = (ph - phk) / dph;
        wp = fmin(fmax(wp, 0.0), 1.0);
        int i1 = o->n[0] > 1 ? i + 1 : i, j1 = o->n[1] > 1 ? j + 1 : j, k1 = (k + 1) % o->n[2];
        double acc[NV] = {0};
        for (int c = 0; c < 8; c++) {
            int ci = (c & 1) ? i1 : i, cj = (c & 2) ? j1 : j, ck = (c & 4) ? k1 : k;
            double f = ((c & 1) ? wr : 1.0 - wr) * ((c & 2) ? wt : 1.0 - wt) * ((c & 4) ? wp : 1.0 - wp);
            double u[NV], wv[NV];
            load(o, o->U, IDX(o, ci, cj, ck), u);
            cons2prim(o, u, wv);
            for (int v = 0; v < NV; v++) acc[v] += f * wv[v];
        }
        double *q = out + (long)p * 13;
        double bmag = sqrt(acc[5] * acc[5] + acc[6] * acc[6] + acc[7] * acc[7]);
        q[0] = tsi;
        q[1] = acc[0] * O_N0;
        q[2] = acc[1] * O_V0;
        q[3] = acc[2] * O_V0;
        q[4] = (acc[3] + o->omega * r * sin(th)) * O_V0;
        q[5] = acc[5] * o->b0; q[6] = acc[6] * o->b0; q[7] = acc[7] * o->b0;
        q[8] = acc[4] * o->p0;
        q[9] = bmag * o->b0;
        q[10] = i; q[11] = j; q[12] = k;
    }
}

/* threads the oracle's OpenMP loops use (timing on the host cores; no effect on the results) */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* the face flux of the configured Riemann solver for primitive face states wl, wr (code units)
 * normal to direction d (test access to one face) */
void orc_riemann(const orc_t *o, const double *wl, const double *wr, int d, double *f)
{
    riemann(o, wl, wr, d, f);
}

