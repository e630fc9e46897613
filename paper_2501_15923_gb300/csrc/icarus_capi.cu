// icarus_capi.cu -- host runtime behind include/icarus.h: context, device memory, grid metrics,
// boundary tables, CUDA-graph replay of the time step, probe ring drain, error reporting.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/icarus.h"
#include "icarus_internal.cuh"
#include "icarus_ops.h"
#include "icarus_ctx.h"

using namespace icarus;

namespace {

// SI constants (CODATA 2018, IAU nominal) and code-unit scales
const double AU = 1.495978707e11, MP = 1.67262192369e-27, KB = 1.380649e-23, MU0 = 1.25663706212e-6,
             GMSUN = 1.32712440018e20, V0 = 1.0e5, N0 = 1.0e6, PI = 3.14159265358979323846;

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail(ICARUS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

// the error of a non-zero status word (bit 0: non-finite state, bit 1: a floor in strict mode)
int status_fail(int status)
{
    if (status & 1) return fail(ICARUS_ENONFINITE, "the solution became non-finite");
    return fail(ICARUS_EFLOOR, "a density or pressure floor acted (options.strict_floors)");
}

}  // namespace

namespace icarus {
// lets other translation units report through icarus_last_error()
int report_error(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace icarus

// struct icarus_ctx is defined in icarus_ctx.h

namespace {

void *dalloc(icarus_ctx *c, size_t bytes)
{
    bytes = (bytes + 255) & ~(size_t)255;
    void *p = nullptr;
    if (c->opts.alloc) p = c->opts.alloc(bytes, c->opts.alloc_user);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (p) c->allocs.push_back(p);
    return p;
}

}  // namespace

void *icarus::ctx_alloc(icarus_ctx *c, size_t bytes) { return dalloc(c, bytes); }

namespace {

// boundary maps [n_maps][5][n2 n3] from SI to code units: field f scaled by s[f] (the same IEEE
// products as a host loop would form)
__global__ void k_maps_to_code(const double *__restrict__ raw, double *__restrict__ out, long long per, long long n,
                               double s0, double s1, double s2, double s3, double s4)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int f = (int)((i / per) % 5);
    const double s = f == 0 ? s0 : (f == 1 ? s1 : (f == 2 ? s2 : (f == 3 ? s3 : s4)));
    out[i] = raw[i] * s;
}

// the FP64 flux's square root and reciprocal beside the library's, element by element:
// y[4i .. 4i + 3] = sqrt_nr, sqrt, rcp_nr, 1 / x
__global__ void k_math_check(const double *x, double *y, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        y[4 * i] = sqrt_nr(x[i]);
        y[4 * i + 1] = sqrt(x[i]);
        y[4 * i + 2] = rcp_nr(x[i]);
        y[4 * i + 3] = 1.0 / x[i];
    }
}

}  // namespace

namespace {

void dfree_all(icarus_ctx *c)
{
    for (void *p : c->allocs) {
        if (c->opts.free) c->opts.free(p, c->opts.alloc_user);
        else if (!c->opts.alloc) cudaFree(p);
    }
    c->allocs.clear();
}

void drop_graph(icarus_ctx *c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    c->p_version++;
}

// radial edge i of a grid with a refined band: in the coordinate u (ln r when stretched, else r)
// the cell density is band_refine inside the band and 1 outside, and edge i is where its integral
// from the inner edge reaches i / n1 of the total (ghost edges continue the outer spacing)
double band_edge(const icarus_grid &g, int i)
{
    return band_edge_at(g.n1, g.x1min, g.x1max, g.band_lo, g.band_hi, g.band_refine,
                        g.geometry == ICARUS_GEOM_SPHERICAL && g.stretch, i);
}

// edges of direction d at padded edge index e (cell i has lower edge i, i in [-2, n+2])
double edge(const icarus_grid &g, int d, int i)
{
    if (d == 0 && g.band_refine > 1) return band_edge(g, i);
    const int n = d == 0 ? g.n1 : (d == 1 ? g.n2 : g.n3);
    const double lo = d == 0 ? g.x1min : (d == 1 ? g.x2min : g.x3min);
    const double hi = d == 0 ? g.x1max : (d == 1 ? g.x2max : g.x3max);
    if (g.geometry == ICARUS_GEOM_SPHERICAL && d == 0 && g.stretch) return lo * pow(hi / lo, (double)i / n);
    return lo + i * ((hi - lo) / n);
}

// host-side metric tables (double), uploaded once; see Metrics for the meaning of each array
int build_metrics(icarus_ctx *c)
{
    const icarus_grid &g = c->grid;
    const Params &P = c->P;
    const bool sph = g.geometry == ICARUS_GEOM_SPHERICAL;
    const int p1 = P.p1, p2 = P.p2, p3 = P.p3;
    std::vector<double> e1(p1 + 1), e2(p2 + 1), e3(p3 + 1);
    for (int i = 0; i <= p1; ++i) e1[i] = edge(g, 0, i - NG);
    for (int j = 0; j <= p2; ++j) e2[j] = edge(g, 1, j - NG);
    for (int k = 0; k <= p3; ++k) e3[k] = edge(g, 2, k - NG);
    auto ctr = [](const std::vector<double> &e, int i) { return 0.5 * (e[i] + e[i + 1]); };
    const double d2 = (g.x2max - g.x2min) / g.n2, d3 = (g.x3max - g.x3min) / g.n3;
    // layout of the single metric buffer
    std::vector<double> buf;
    std::vector<size_t> off;
    auto push = [&](const std::vector<double> &v) { off.push_back(buf.size()); buf.insert(buf.end(), v.begin(), v.end()); };
    std::vector<double> x1c(p1), a1(p1 + 1), iv1(p1), q1(p1), gp1(p1), iw1(p1), ih2(p1), ig1(p1), gmr2(p1);
    for (int i = 0; i <= p1; ++i) a1[i] = sph ? e1[i] * e1[i] : 1.0;
    for (int i = 0; i < p1; ++i) {
        double rm = e1[i], rp = e1[i + 1];
        x1c[i] = ctr(e1, i);
        double v1 = sph ? (rp * rp * rp - rm * rm * rm) / 3.0 : (rp - rm);
        iv1[i] = 1.0 / v1;
        q1[i] = sph ? 0.5 * (rp * rp - rm * rm) / v1 : 1.0;
        iw1[i] = 1.0 / (rp - rm);
        ih2[i] = sph ? 1.0 / x1c[i] : 1.0;
        gmr2[i] = sph ? c->gm_code / (x1c[i] * x1c[i]) : 0.0;
    }
    for (int i = 0; i < p1; ++i) {
        gp1[i] = (a1[i + 1] - a1[i]) * iv1[i];
        double xm = i > 0 ? x1c[i - 1] : x1c[i] - (x1c[i + 1] - x1c[i]);
        double xp = i + 1 < p1 ? x1c[i + 1] : x1c[i] + (x1c[i] - x1c[i - 1]);
        ig1[i] = 1.0 / (xp - xm);
    }
    std::vector<double> x2c(p2), a2(p2 + 1), iv2(p2), q2(p2), gq2(p2), sn(p2), cs(p2), ct(p2), is3(p2), ig2(p2);
    for (int j = 0; j <= p2; ++j) a2[j] = sph ? sin(e2[j]) : 1.0;
    for (int j = 0; j < p2; ++j) {
        x2c[j] = ctr(e2, j);
        double v2 = sph ? (cos(e2[j]) - cos(e2[j + 1])) : (e2[j + 1] - e2[j]);
        iv2[j] = 1.0 / v2;
        q2[j] = sph ? (e2[j + 1] - e2[j]) / v2 : 1.0;
        gq2[j] = sph ? (a2[j + 1] - a2[j]) / v2 : 0.0;
        sn[j] = sph ? sin(x2c[j]) : 1.0;
        cs[j] = sph ? cos(x2c[j]) : 0.0;
        ct[j] = sph ? cos(x2c[j]) / sin(x2c[j]) : 0.0;
        is3[j] = sph ? 1.0 / sin(x2c[j]) : 1.0;
    }
    for (int j = 0; j < p2; ++j) {
        double xm = j > 0 ? x2c[j - 1] : x2c[j] - d2;
        double xp = j + 1 < p2 ? x2c[j + 1] : x2c[j] + d2;
        ig2[j] = 1.0 / (xp - xm);
    }
    std::vector<double> x3c(p3), ig3(p3);
    for (int k = 0; k < p3; ++k) x3c[k] = ctr(e3, k);
    for (int k = 0; k < p3; ++k) {
        double xm = k > 0 ? x3c[k - 1] : x3c[k] - d3;
        double xp = k + 1 < p3 ? x3c[k + 1] : x3c[k] + d3;
        ig3[k] = 1.0 / (xp - xm);
    }
    // CME footprint unit vectors of the boundary columns [3][n2][n3]
    std::vector<double> col(3 * (size_t)g.n2 * g.n3);
    const size_t per = (size_t)g.n2 * g.n3;
    for (int j = 0; j < g.n2; ++j)
        for (int k = 0; k < g.n3; ++k) {
            double th = x2c[j + NG], ph = x3c[k + NG];
            col[j * g.n3 + k] = sin(th) * cos(ph);
            col[per + j * g.n3 + k] = sin(th) * sin(ph);
            col[2 * per + j * g.n3 + k] = cos(th);
        }
    std::vector<double> ldx2((size_t)p1 * p2);
    for (int j = 0; j < p2; ++j)
        for (int i = 0; i < p1; ++i) {
            const double w1 = iw1[i], w2 = ih2[i] * (1.0 / d2), w3 = ih2[i] * is3[j] * (1.0 / d3);
            ldx2[(size_t)j * p1 + i] = 1.0 / (w1 * w1 + w2 * w2 + w3 * w3);
        }
    // per-cell products of the per-axis factors (the FP64 update and div B read them); each formed
    // in the order the device formed it before, so the values are the same
    const double iv3 = 1.0 / d3, opts_divb_coef = P.divb_coef;
    const size_t ncf = (size_t)p1 * p2;
    std::vector<double> cf((size_t)CF_N * ncf);
    for (int j = 0; j < p2; ++j)
        for (int i = 0; i < p1; ++i) {
            const size_t q = (size_t)j * p1 + i;
            const double jv = q1[i] * iv2[j];
            cf[CF_AM * ncf + q] = a1[i] * iv1[i];
            cf[CF_AP * ncf + q] = a1[i + 1] * iv1[i];
            cf[CF_BM * ncf + q] = a2[j] * jv;
            cf[CF_BP * ncf + q] = a2[j + 1] * jv;
            cf[CF_KV * ncf + q] = q1[i] * q2[j] * iv3;
            cf[CF_Q1GQ2 * ncf + q] = q1[i] * gq2[j];
            cf[CF_IH2IG2 * ncf + q] = ih2[i] * ig2[j];
            cf[CF_IH2IS3 * ncf + q] = ih2[i] * is3[j];
            cf[CF_JV * ncf + q] = jv;
            cf[CF_ORS * ncf + q] = P.omega * x1c[i] * sn[j];
            const double ld = opts_divb_coef * ldx2[q];
            cf[CF_LD0 * ncf + q] = ld * ig1[i];
            cf[CF_LD1 * ncf + q] = ld * (ih2[i] * ig2[j]);
            cf[CF_LD2 * ncf + q] = ld * (ih2[i] * is3[j]);
        }
    push(x1c); push(a1); push(iv1); push(q1); push(gp1); push(iw1); push(ih2); push(ig1); push(gmr2);
    push(x2c); push(a2); push(iv2); push(q2); push(gq2); push(sn); push(cs); push(ct); push(is3); push(ig2);
    push(x3c); push(ig3); push(col); push(ldx2); push(cf);
    c->metric = (double *)dalloc(c, buf.size() * sizeof(double));
    if (!c->metric) return fail(ICARUS_ENOMEM, "metric allocation failed");
    CK(cudaMemcpyAsync(c->metric, buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    // the same tables rounded to float, for the single-precision arithmetic
    std::vector<float> fbuf(buf.begin(), buf.end());
    float *mfb = (float *)dalloc(c, fbuf.size() * sizeof(float));
    if (!mfb) return fail(ICARUS_ENOMEM, "metric allocation failed");
    CK(cudaMemcpyAsync(mfb, fbuf.data(), fbuf.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    auto bind = [&](auto &m, const auto *b) {
        int q = 0;
        m.x1c = b + off[q++]; m.a1 = b + off[q++]; m.iv1 = b + off[q++]; m.q1 = b + off[q++]; m.gp1 = b + off[q++];
        m.iw1 = b + off[q++]; m.ih2 = b + off[q++]; m.ig1 = b + off[q++]; m.gm_r2 = b + off[q++];
        m.x2c = b + off[q++]; m.a2 = b + off[q++]; m.iv2 = b + off[q++]; m.q2 = b + off[q++]; m.gq2 = b + off[q++];
        m.sn = b + off[q++]; m.cs = b + off[q++]; m.ct = b + off[q++]; m.is3 = b + off[q++]; m.ig2 = b + off[q++];
        m.x3c = b + off[q++]; m.ig3 = b + off[q++]; m.colvec = b + off[q++]; m.ldx2 = b + off[q++];
        m.cf = b + off[q++];
        m.cf_p1 = p1;
        m.cf_n = (long long)ncf;
    };
    Metrics &m = c->P.m;
    bind(m, (const double *)c->metric);
    m.d2 = d2; m.d3 = d3;
    m.id2 = 1.0 / d2; m.id3 = 1.0 / d3;
    m.iv3 = 1.0 / d3;
    MetricsT<float> &mf = c->P.mf;
    bind(mf, (const float *)mfb);
    mf.d2 = (float)m.d2; mf.d3 = (float)m.d3; mf.id2 = (float)m.id2; mf.id3 = (float)m.id3; mf.iv3 = (float)m.iv3;
    // smallest interior cell width (dr, r dtheta, r sin(theta) dphi on the sphere): the GLM c_h
    double dmin = 1e300;
    for (int k = NG; k < NG + g.n3; ++k)
        for (int j = NG; j < NG + g.n2; ++j)
            for (int i = NG; i < NG + g.n1; ++i) {
                const double w1 = e1[i + 1] - e1[i], w2 = e2[j + 1] - e2[j], w3 = e3[k + 1] - e3[k];
                if (sph) {
                    const double rc = ctr(e1, i);
                    dmin = fmin(dmin, fmin(w1, fmin(rc * w2, rc * sin(ctr(e2, j)) * w3)));
                } else {
                    dmin = fmin(dmin, fmin(w1, fmin(w2, w3)));
                }
            }
    c->P.glm_dmin = dmin;
    return ICARUS_OK;
}

// the whole-stage fused kernel (options.fused = 1)
bool use_fused_stage(const icarus_ctx *c) { return c->ops.fused_stage && c->opts.fused == 1; }

// the update with the r-face fluxes inside it, the default (options.fused = 0) where the precision
// form has it (FP32, MIXED) and the options allow it (TVDLF / HLL, no GLM, no tracer: the tracer
// reads the r mass fluxes); options.fused = 2 keeps the separate r-flux kernel
bool use_update_rf(const icarus_ctx *c)
{
    return c->ops.update_rf && c->opts.fused == 0 && c->opts.flux != ICARUS_FLUX_HLLD &&
           c->opts.divb != ICARUS_DIVB_GLM && !c->opts.tracer;
}

void enqueue_step(icarus_ctx *c, cudaStream_t s)
{
    const Params &P = c->P;
    if (use_fused_stage(c)) {
        c->ops.fill_ghosts(P, c->U, c->W, 1, s);
        c->ops.fused_stage(P, 1, c->U, c->W, c->U1, c->W1, s);
        c->ops.fill_ghosts(P, c->U1, c->W1, 2, s);
        c->ops.fused_stage(P, 2, c->U1, c->W1, c->U, c->W, s);
        if (P.n_probes > 0) c->ops.probe(P, c->W, s);
        return;
    }
    // stage 1: U, W at t  ->  U1, W1 (tracer: rho c in T, c in C  ->  T1, C1, with the stage's mass fluxes)
    // (GLM: psi in Psi -> Psi1 -> Psi, its (B_n, psi) face states after the MHD fluxes)
    const bool tr = c->opts.tracer != 0, glm = P.divb == ICARUS_DIVB_GLM, rf = use_update_rf(c);
    c->ops.fill_ghosts(P, c->U, c->W, 1, s);
    if (tr) c->ops.tracer_ghost(P, c->C, 1, s);
    if (glm) c->ops.glm_ghost(P, c->Psi, s);
    if (glm) c->ops.fluxes_glm(P, c->W, c->Psi, c->F1, c->F2, c->F3, c->FP1, c->FP2, c->FP3, s);
    else if (rf) { c->ops.flux_dir(P, 1, c->W, c->F2, s); c->ops.flux_dir(P, 2, c->W, c->F3, s); }
    else c->ops.fluxes(P, c->W, c->F1, c->F2, c->F3, s);
    if (P.divb == 1 || P.divb == 3) c->ops.divb(P, c->W, c->divB, s);
    if (rf) c->ops.update_rf(P, 1, c->U, c->W, c->U1, c->W1, c->F2, c->F3, c->divB, s);
    else c->ops.update(P, 1, c->U, c->W, c->U1, c->W1, c->F1, c->F2, c->F3, c->divB, s);
    if (glm) c->ops.glm_update(P, 1, c->Psi, c->Psi1, c->FP1, c->FP2, c->FP3, s);
    if (tr) c->ops.tracer_update(P, 1, c->C, c->F1, c->F2, c->F3, c->T, c->T1, c->U1, c->C1, s);
    // stage 2: U1, W1 at t + dt  ->  U, W (in place), next dt, t += dt
    c->ops.fill_ghosts(P, c->U1, c->W1, 2, s);
    if (tr) c->ops.tracer_ghost(P, c->C1, 2, s);
    if (glm) c->ops.glm_ghost(P, c->Psi1, s);
    if (glm) c->ops.fluxes_glm(P, c->W1, c->Psi1, c->F1, c->F2, c->F3, c->FP1, c->FP2, c->FP3, s);
    else if (rf) { c->ops.flux_dir(P, 1, c->W1, c->F2, s); c->ops.flux_dir(P, 2, c->W1, c->F3, s); }
    else c->ops.fluxes(P, c->W1, c->F1, c->F2, c->F3, s);
    if (P.divb == 1 || P.divb == 3) c->ops.divb(P, c->W1, c->divB, s);
    if (rf) c->ops.update_rf(P, 2, c->U1, c->W1, c->U, c->W, c->F2, c->F3, c->divB, s);
    else c->ops.update(P, 2, c->U1, c->W1, c->U, c->W, c->F1, c->F2, c->F3, c->divB, s);
    if (glm) c->ops.glm_update(P, 2, c->Psi1, c->Psi, c->FP1, c->FP2, c->FP3, s);
    if (tr) c->ops.tracer_update(P, 2, c->C1, c->F1, c->F2, c->F3, c->T1, c->T, c->U, c->C, s);
    if (P.n_probes > 0) c->ops.probe(P, c->W, s);
}

int count_launches(const icarus_ctx *c)
{
    int per_stage = use_fused_stage(c) ? 3 + 1
                  : 3 + (use_update_rf(c) ? 2 : 3) + (c->P.divb == 1 || c->P.divb == 3 ? 1 : 0) + 1 +
                        (c->opts.tracer ? 2 : 0) +
                        (c->P.divb == ICARUS_DIVB_GLM ? 2 : 0);
    return 2 * per_stage + (c->P.n_probes > 0 ? 1 : 0);
}

int build_graph(icarus_ctx *c)
{
    drop_graph(c);
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    enqueue_step(c, c->stream);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess) return fail(ICARUS_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ICARUS_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    c->launches_per_step = count_launches(c);
    return ICARUS_OK;
}

int first_dt(icarus_ctx *c)
{
    c->ops.fill_ghosts(c->P, c->U, c->W, 1, c->stream);
    c->ops.cfl(c->P, c->W, c->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    return ICARUS_OK;
}

}  // namespace

namespace icarus {
// one time step of the context enqueued on stream s (the batched form captures members' steps on
// parallel streams into one graph)
void enqueue_step_on(icarus_ctx *c, cudaStream_t s) { enqueue_step(c, s); }

// the grids every entry point that takes an icarus_grid accepts (EINVAL with a message otherwise)
int check_grid(const icarus_grid *g)
{
    if (g->n1 < 1 || g->n2 < 1 || g->n3 < 1) return fail(ICARUS_EINVAL, "cell counts must be >= 1");
    if ((long long)(g->n1 + 4) * (g->n2 + 4) * (g->n3 + 4) > (1LL << 31))
        return fail(ICARUS_EINVAL, "grid too large (padded cells must fit in 2^31)");
    if (g->geometry != ICARUS_GEOM_SPHERICAL && g->geometry != ICARUS_GEOM_CARTESIAN)
        return fail(ICARUS_EINVAL, "unknown geometry %d", g->geometry);
    if (!(g->x1max > g->x1min) || !(g->x2max > g->x2min) || !(g->x3max > g->x3min))
        return fail(ICARUS_EINVAL, "empty coordinate range");
    if (g->band_refine < 0 || g->band_refine > 64) return fail(ICARUS_EINVAL, "band_refine must be in [0, 64]");
    if (g->band_refine > 1 && !(g->x1min < g->band_lo && g->band_lo < g->band_hi && g->band_hi < g->x1max))
        return fail(ICARUS_EINVAL, "the refined band must lie strictly inside (x1min, x1max)");
    if (g->geometry == ICARUS_GEOM_SPHERICAL) {
        if (!(g->x1min > 0)) return fail(ICARUS_EINVAL, "r_in must be > 0");
        double d2 = (g->x2max - g->x2min) / g->n2;
        if (!(g->x2min - 2 * d2 > 0) || !(g->x2max + 2 * d2 < PI))
            return fail(ICARUS_EINVAL, "colatitude range with its ghost cells must stay inside (0, pi)");
    }
    for (int s = 0; s < 6; ++s) {
        int b = g->bc[s];
        if (b < 0 || b > 3) return fail(ICARUS_EINVAL, "bad boundary code %d on face %d", b, s);
        if (b == ICARUS_BC_DRIVEN && (s != 0 || g->geometry != ICARUS_GEOM_SPHERICAL))
            return fail(ICARUS_EINVAL, "DRIVEN is only valid on the inner radial face of a spherical grid");
        int n = s < 2 ? g->n1 : (s < 4 ? g->n2 : g->n3);
        if (b == ICARUS_BC_REFLECT && n < 2) return fail(ICARUS_EINVAL, "REFLECT needs >= 2 cells");
    }
    return ICARUS_OK;
}
}  // namespace icarus

extern "C" {

const char *icarus_last_error(void) { return g_err.c_str(); }

int icarus_init(const icarus_grid *grid, double gamma, double omega_rot, const icarus_options *opts, icarus_ctx **out)
{
    if (!grid || !opts || !out) return fail(ICARUS_EINVAL, "NULL argument");
    int rc = check_grid(grid);
    if (rc) return rc;
    if (!(gamma > 1.0)) return fail(ICARUS_EINVAL, "gamma must be > 1");
    if (!(opts->cfl > 0.0 && opts->cfl <= 1.0)) return fail(ICARUS_EINVAL, "cfl must be in (0, 1]");
    if (opts->limiter < 0 || opts->limiter > 2 || opts->flux < 0 || opts->flux > 2 || opts->divb < 0 || opts->divb > 3 ||
        opts->init_vphi < 0 || opts->init_vphi > 1 || opts->cme_model < 0 || opts->cme_model > 1 ||
        opts->tracer < 0 || opts->tracer > 1 || opts->strict_floors < 0 || opts->strict_floors > 1)
        return fail(ICARUS_EINVAL, "bad limiter / flux / divb / init_vphi / cme_model / tracer / strict_floors option");
    if (opts->precision < 0 || opts->precision > 2) return fail(ICARUS_EINVAL, "bad precision");
    if (opts->fused < 0 || opts->fused > 2) return fail(ICARUS_EINVAL, "bad fused option (0, 1 or 2)");
    if (opts->fused == 1 && opts->flux == ICARUS_FLUX_HLLD)
        return fail(ICARUS_EINVAL, "the fused stage kernel supports the TVDLF and HLL fluxes only");
    if (opts->fused == 1 && opts->tracer) return fail(ICARUS_EINVAL, "the fused stage kernel carries no CME tracer");
    if (opts->divb == ICARUS_DIVB_GLM && opts->fused == 1)
        return fail(ICARUS_EINVAL, "GLM div-B control runs with the separate kernels, not the fused stage");
    if (opts->divb == ICARUS_DIVB_POWELL && opts->fused == 1)
        return fail(ICARUS_EINVAL, "the Powell source runs with the separate kernels, not the fused stage");
    if (opts->divb == ICARUS_DIVB_GLM && !(opts->glm_alpha >= 0.0)) return fail(ICARUS_EINVAL, "glm_alpha must be >= 0");
    if (opts->ring_capacity < 1) return fail(ICARUS_EINVAL, "ring_capacity must be >= 1");
    icarus_ctx *c = new icarus_ctx();
    c->grid = *grid;
    c->opts = *opts;
    c->ops = opts->precision == ICARUS_FP64 ? ops_fp64() : (opts->precision == ICARUS_FP32 ? ops_fp32() : ops_mixed());
    if (opts->cuda_stream) c->stream = (cudaStream_t)opts->cuda_stream;
    else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(ICARUS_ECUDA, "stream creation failed");
        }
        c->own_stream = true;
    }
    Params &P = c->P;
    P.n1 = grid->n1; P.n2 = grid->n2; P.n3 = grid->n3;
    P.p1 = P.n1 + 2 * NG; P.p2 = P.n2 + 2 * NG; P.p3 = P.n3 + 2 * NG;
    P.nt = (long long)P.p1 * P.p2 * P.p3;
    P.geom = grid->geometry;
    for (int s = 0; s < 6; ++s) P.bc[s] = grid->bc[s];
    P.limiter = opts->limiter; P.flux = opts->flux; P.gravity = opts->gravity; P.divb = opts->divb;
    P.init_vphi = opts->init_vphi;
    P.cme_model = opts->cme_model;
    P.r_in = grid->x1min;
    P.gamma = gamma;
    P.divb_coef = opts->divb_coef; P.rho_floor = opts->rho_floor; P.p_floor = opts->p_floor;
    P.glm_alpha = opts->glm_alpha;
    P.strict_floors = opts->strict_floors;
    c->t0 = AU / V0;
    const double rho0 = MP * N0;
    c->p0 = rho0 * V0 * V0;
    c->b0 = sqrt(MU0 * rho0) * V0;
    c->omega_code = grid->geometry == ICARUS_GEOM_SPHERICAL ? omega_rot * c->t0 : 0.0;
    c->gm_code = GMSUN / (AU * V0 * V0);
    if (grid->geometry != ICARUS_GEOM_SPHERICAL) P.gravity = 0;
    P.omega = c->omega_code;
    P.omega_si = grid->geometry == ICARUS_GEOM_SPHERICAL ? omega_rot : 0.0;
    P.t0 = c->t0; P.b0 = c->b0; P.p0 = c->p0;
    P.ph = PhysT<double>{P.gamma, P.gamma - 1.0, 1.0 / (P.gamma - 1.0), P.omega, P.divb_coef, P.rho_floor, P.p_floor};
    P.phf = PhysT<float>{(float)P.ph.gamma, (float)P.ph.gm1, (float)P.ph.igm1, (float)P.ph.omega,
                         (float)P.ph.divb_coef, (float)P.ph.rho_floor, (float)P.ph.p_floor};
    P.ring_cap = opts->ring_capacity;
    rc = build_metrics(c);
    if (rc) { icarus_destroy(c); return rc; }
    const size_t nt = P.nt, ts = c->ops.ts_size, tw = c->ops.tw_size;
    c->U = dalloc(c, NV * nt * ts);
    c->U1 = dalloc(c, NV * nt * ts);
    c->W = dalloc(c, NV * nt * tw);
    c->W1 = dalloc(c, NV * nt * tw);
    c->F1 = dalloc(c, NV * (size_t)P.n3 * P.n2 * (P.n1 + 1) * tw);
    c->F2 = dalloc(c, NV * (size_t)P.n3 * (P.n2 + 1) * P.n1 * tw);
    c->F3 = dalloc(c, NV * (size_t)(P.n3 + 1) * P.n2 * P.n1 * tw);
    c->divB = dalloc(c, nt * tw);
    const long long ncell = (long long)P.n1 * P.n2 * P.n3;
    c->sc = (Scalars *)dalloc(c, sizeof(Scalars));
    c->stage_buf = (double *)dalloc(c, NV * (size_t)ncell * sizeof(double));
    if (opts->divb == ICARUS_DIVB_GLM) {
        c->Psi = dalloc(c, nt * ts);
        c->Psi1 = dalloc(c, nt * ts);
        c->FP1 = dalloc(c, (size_t)P.n3 * P.n2 * (P.n1 + 1) * tw);
        c->FP2 = dalloc(c, (size_t)P.n3 * (P.n2 + 1) * P.n1 * tw);
        c->FP3 = dalloc(c, (size_t)(P.n3 + 1) * P.n2 * P.n1 * tw);
        if (!c->Psi || !c->Psi1 || !c->FP1 || !c->FP2 || !c->FP3) {
            icarus_destroy(c);
            return fail(ICARUS_ENOMEM, "device allocation failed");
        }
        CK(cudaMemsetAsync(c->Psi, 0, nt * ts, c->stream));
        CK(cudaMemsetAsync(c->Psi1, 0, nt * ts, c->stream));
        P.psi0 = c->Psi;
        P.psi1 = c->Psi1;
    }
    if (opts->tracer) {
        c->T = dalloc(c, nt * ts);
        c->T1 = dalloc(c, nt * ts);
        c->C = dalloc(c, nt * tw);
        c->C1 = dalloc(c, nt * tw);
        if (!c->T || !c->T1 || !c->C || !c->C1) {
            icarus_destroy(c);
            return fail(ICARUS_ENOMEM, "device allocation failed");
        }
        CK(cudaMemsetAsync(c->T, 0, nt * ts, c->stream));
        CK(cudaMemsetAsync(c->T1, 0, nt * ts, c->stream));
        CK(cudaMemsetAsync(c->C, 0, nt * tw, c->stream));
        CK(cudaMemsetAsync(c->C1, 0, nt * tw, c->stream));
    }
    if (!c->U || !c->U1 || !c->W || !c->W1 || !c->F1 || !c->F2 || !c->F3 || !c->divB || !c->sc || !c->stage_buf) {
        icarus_destroy(c);
        return fail(ICARUS_ENOMEM, "device allocation failed");
    }
    P.sc = c->sc;
    // host-mapped status word: each step's last kernel copies the status there, so icarus_step can
    // report it without synchronising
    if (cudaHostAlloc((void **)&c->hstatus, sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
        c->hstatus = nullptr;
        icarus_destroy(c);
        return fail(ICARUS_ENOMEM, "host-mapped status allocation failed");
    }
    *(volatile int *)c->hstatus = 0;
    CK(cudaHostGetDevicePointer((void **)&P.hstatus, c->hstatus, 0));
    Scalars s0{};
    s0.cfl = opts->cfl;
    CK(cudaMemsetAsync(c->U, 0, NV * nt * ts, c->stream));
    CK(cudaMemsetAsync(c->U1, 0, NV * nt * ts, c->stream));
    CK(cudaMemsetAsync(c->W, 0, NV * nt * tw, c->stream));
    CK(cudaMemsetAsync(c->W1, 0, NV * nt * tw, c->stream));
    CK(cudaMemsetAsync(c->divB, 0, nt * tw, c->stream));
    CK(cudaMemcpyAsync(c->sc, &s0, sizeof s0, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *out = c;
    return ICARUS_OK;
}

int icarus_set_boundary(icarus_ctx *c, int n_maps, const double *t_maps, const double *maps, int n_cme, const double *cmes)
{
    if (!c) return fail(ICARUS_EINVAL, "NULL context");
    if (n_maps < 1 || !t_maps || !maps) return fail(ICARUS_EINVAL, "need n_maps >= 1 maps with their times");
    if (n_cme < 0 || (n_cme > 0 && !cmes)) return fail(ICARUS_EINVAL, "bad CME table");
    for (int m = 1; m < n_maps; ++m)
        if (!(t_maps[m] > t_maps[m - 1])) return fail(ICARUS_EINVAL, "map times must increase");
    Params &P = c->P;
    const size_t per = (size_t)P.n2 * P.n3;
    const size_t nm = (size_t)n_maps * 5 * per, nc = 10 * (size_t)(n_cme > 0 ? n_cme : 1);
    // the previous tables may still be in flight from the staging buffer or in use on the device
    CK(cudaStreamSynchronize(c->stream));
    // the small tables (map times, CME rows) in code units, written into pinned host memory
    std::vector<double> fallback;
    double *hs = nullptr;
    if (n_maps + nc > c->hstage_cap) {
        if (c->hstage) cudaFreeHost(c->hstage);
        c->hstage = nullptr;
        c->hstage_cap = 0;
        if (cudaHostAlloc((void **)&c->hstage, (n_maps + nc) * sizeof(double), cudaHostAllocDefault) == cudaSuccess)
            c->hstage_cap = n_maps + nc;
        else {
            c->hstage = nullptr;
            cudaGetLastError();
        }
    }
    if (c->hstage) hs = c->hstage;
    else {
        fallback.resize(n_maps + nc);
        hs = fallback.data();
    }
    double *ht = hs, *hc = ht + n_maps;
    for (int m = 0; m < n_maps; ++m) ht[m] = t_maps[m] / c->t0;
    for (size_t q = 0; q < nc; ++q) hc[q] = 0.0;
    for (int q = 0; q < n_cme; ++q) {
        const double *s = cmes + 8 * q;
        double *d = hc + 10 * q;
        d[0] = s[0] / c->t0;
        d[1] = s[1] / c->t0;
        d[2] = cos(s[2]) * cos(s[3]);
        d[3] = cos(s[2]) * sin(s[3]);
        d[4] = sin(s[2]);
        d[5] = cos(s[4]);
        d[6] = s[5] / V0;
        d[7] = s[6] / N0;
        d[8] = 2.0 * s[6] * KB * s[7] / c->p0;
        // spherical cloud: radius in AU, and the crossing time 2 R / v as the window length
        d[9] = c->grid.x1min * sin(s[4]);
        if (c->P.cme_model == ICARUS_CME_SPHERE) d[1] = 2.0 * d[9] / d[6];
    }
    if (nm > c->maps_cap || (size_t)n_maps > c->tmaps_cap) {
        c->maps = (double *)dalloc(c, nm * sizeof(double));
        c->tmaps = (double *)dalloc(c, n_maps * sizeof(double));
        if (!c->maps || !c->tmaps) return fail(ICARUS_ENOMEM, "map allocation failed");
        c->maps_cap = nm;
        c->tmaps_cap = n_maps;
    }
    if (nm > c->maps_raw_cap) {
        c->maps_raw = (double *)dalloc(c, nm * sizeof(double));
        if (!c->maps_raw) return fail(ICARUS_ENOMEM, "map allocation failed");
        c->maps_raw_cap = nm;
    }
    if (nc > c->cme_cap) {
        c->cme = (double *)dalloc(c, nc * sizeof(double));
        if (!c->cme) return fail(ICARUS_ENOMEM, "CME allocation failed");
        c->cme_cap = nc;
    }
    // the maps as given (one DMA when the caller's array is pinned), then scaled on the device; all
    // in stream order after the steps already queued, which may still read the previous tables
    CK(cudaMemcpyAsync(c->maps_raw, maps, nm * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    k_maps_to_code<<<(unsigned int)((nm + 255) / 256), 256, 0, c->stream>>>(c->maps_raw, c->maps, (long long)per,
                                                                             (long long)nm, 1.0 / V0, 1.0 / N0,
                                                                             1.0 / c->p0, 1.0 / c->b0, 1.0 / c->b0);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c->tmaps, ht, n_maps * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->cme, hc, nc * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    // the captured step reads the tables through these pointers and counts: a new graph only when
    // one of them changes
    if (P.maps != c->maps || P.t_maps != c->tmaps || P.cme != c->cme || P.n_maps != n_maps || P.n_cme != n_cme)
        drop_graph(c);
    P.maps = c->maps; P.t_maps = c->tmaps; P.cme = c->cme;
    P.n_maps = n_maps; P.n_cme = n_cme;
    c->have_boundary = true;
    if (!c->have_state) {
        if (c->grid.geometry != ICARUS_GEOM_SPHERICAL) return fail(ICARUS_EINVAL, "initial state from maps needs a spherical grid");
        c->ops.init_state(P, c->U, c->W, c->grid.x1min, c->stream);
        CK(cudaGetLastError());
        c->have_state = true;
        int rc = first_dt(c);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(c->stream));
    return ICARUS_OK;
}

int icarus_step(icarus_ctx *c, int n)
{
    if (!c) return fail(ICARUS_EINVAL, "NULL context");
    if (n < 0) return fail(ICARUS_EINVAL, "n must be >= 0");
    if (!c->have_state) return fail(ICARUS_ESTATE, "no state: call icarus_set_boundary or icarus_set_state first");
    if (c->grid.bc[0] == ICARUS_BC_DRIVEN && !c->have_boundary) return fail(ICARUS_ESTATE, "DRIVEN boundary without maps");
    // sticky status of the steps completed so far (host-mapped copy; no synchronisation)
    if (c->hstatus) {
        const int st = *(volatile int *)c->hstatus;
        if (st) return status_fail(st);
    }
    if (!c->graph) {
        int rc = build_graph(c);
        if (rc) return rc;
    }
    for (int q = 0; q < n; ++q) CK(cudaGraphLaunch(c->graph, c->stream));
    return ICARUS_OK;
}

int icarus_step_recover(icarus_ctx *c, int n, int max_retries, int *halvings)
{
    if (halvings) *halvings = 0;
    if (n < 0) return fail(ICARUS_EINVAL, "n must be >= 0");
    if (max_retries < 0 || max_retries > 20) return fail(ICARUS_EINVAL, "max_retries must be in [0, 20]");
    if (!c) return fail(ICARUS_EINVAL, "NULL context");
    if (!c->have_state) return fail(ICARUS_ESTATE, "no state: call icarus_set_boundary or icarus_set_state first");
    if (c->grid.bc[0] == ICARUS_BC_DRIVEN && !c->have_boundary) return fail(ICARUS_ESTATE, "DRIVEN boundary without maps");
    const Params &P = c->P;
    cudaStream_t s = c->stream;
    const size_t nt = P.nt, ts = c->ops.ts_size, tw = c->ops.tw_size;
    const bool tr = c->opts.tracer != 0, glm = P.divb == ICARUS_DIVB_GLM;
    Scalars s0;
    CK(cudaMemcpyAsync(&s0, c->sc, sizeof s0, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (s0.status) return status_fail(s0.status);
    if (n == 0) return ICARUS_OK;
    if (!c->snapU) {
        c->snapU = dalloc(c, NV * nt * ts);
        if (tr) { c->snapT = dalloc(c, nt * ts); c->snapC = dalloc(c, nt * tw); }
        if (glm) c->snapPsi = dalloc(c, nt * ts);
        if (!c->snapU || (tr && (!c->snapT || !c->snapC)) || (glm && !c->snapPsi)) {
            c->snapU = c->snapT = c->snapC = c->snapPsi = nullptr;   // the allocations stay tracked
            return fail(ICARUS_ENOMEM, "snapshot allocation failed");
        }
    }
    // the snapshot: the padded state (the primitives are rebuilt from it), tracer, psi; the
    // scalars (time, dt, ring head, floor count) stay in s0 on the host
    CK(cudaMemcpyAsync(c->snapU, c->U, NV * nt * ts, cudaMemcpyDeviceToDevice, s));
    if (tr) {
        CK(cudaMemcpyAsync(c->snapT, c->T, nt * ts, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(c->snapC, c->C, nt * tw, cudaMemcpyDeviceToDevice, s));
    }
    if (glm) CK(cudaMemcpyAsync(c->snapPsi, c->Psi, nt * ts, cudaMemcpyDeviceToDevice, s));
    // put the snapshot back with CFL number cfl and status word status
    auto restore = [&](double cfl, int status) -> int {
        CK(cudaMemcpyAsync(c->U, c->snapU, NV * nt * ts, cudaMemcpyDeviceToDevice, s));
        c->ops.prims(P, c->U, c->W, s);
        if (tr) {
            CK(cudaMemcpyAsync(c->T, c->snapT, nt * ts, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(c->C, c->snapC, nt * tw, cudaMemcpyDeviceToDevice, s));
        }
        if (glm) CK(cudaMemcpyAsync(c->Psi, c->snapPsi, nt * ts, cudaMemcpyDeviceToDevice, s));
        Scalars r = s0;
        r.cfl = cfl;
        r.status = status;
        r.done = 0;
        CK(cudaMemcpyAsync(c->sc, &r, sizeof r, cudaMemcpyHostToDevice, s));
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s));                      // r is on this frame
        if (c->hstatus) *(volatile int *)c->hstatus = status;
        return ICARUS_OK;
    };
    const double cfl0 = s0.cfl;
    double cfl = cfl0;
    int status = 0;
    for (int h = 0; h <= max_retries; ++h) {
        if (h > 0) {
            cfl *= 0.5;
            int rc = restore(cfl, 0);
            if (!rc) rc = first_dt(c);                     // dt of the restored state at the halved CFL
            if (rc) return rc;
        }
        int rc = icarus_step(c, n);
        if (rc) return rc;
        Scalars se;
        CK(cudaMemcpyAsync(&se, c->sc, sizeof se, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        status = se.status;
        if (!status) {
            if (halvings) *halvings = h;
            if (h > 0) {
                // the configured CFL number back, and the next dt with it
                se.cfl = cfl0;
                CK(cudaMemcpyAsync(c->sc, &se, sizeof se, cudaMemcpyHostToDevice, s));
                return first_dt(c);
            }
            return ICARUS_OK;
        }
        if (halvings) *halvings = h;
    }
    int rc = restore(cfl0, status);
    if (rc) return rc;
    return status_fail(status);
}

int icarus_sample(icarus_ctx *c, int n_probes, int n_knots, const double *traj, double *out, int cap, int *n_written)
{
    if (!c) return fail(ICARUS_EINVAL, "NULL context");
    if (traj) {
        if (n_probes < 1 || n_probes > 1024 || n_knots < 1) return fail(ICARUS_EINVAL, "need 1..1024 probes and >= 1 knot");
        if (!c->have_state) return fail(ICARUS_ESTATE, "no state to sample");
        size_t tn = (size_t)n_probes * n_knots * 4;
        CK(cudaStreamSynchronize(c->stream));
        if (tn > c->traj_cap) {
            c->traj = (double *)dalloc(c, tn * sizeof(double));
            if (!c->traj) return fail(ICARUS_ENOMEM, "trajectory allocation failed");
            c->traj_cap = tn;
        }
        if (n_probes != c->P.n_probes || !c->ring) {
            c->ring = (double *)dalloc(c, (size_t)c->P.ring_cap * n_probes * IC_NPROBE_REC * sizeof(double));
            if (!c->ring) return fail(ICARUS_ENOMEM, "ring allocation failed");
        }
        CK(cudaMemcpyAsync(c->traj, traj, tn * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        // a new registration starts an empty ring
        long long head = 0;
        CK(cudaMemcpyAsync(&c->sc->ring_head, &head, sizeof head, cudaMemcpyHostToDevice, c->stream));
        c->ring_tail = 0;
        c->P.traj = c->traj; c->P.ring = c->ring;
        c->P.n_probes = n_probes; c->P.n_knots = n_knots;
        drop_graph(c);
        c->ops.probe(c->P, c->W, c->stream);
        CK(cudaGetLastError());
    }
    if (n_written) *n_written = 0;
    if (c->P.n_probes == 0) return ICARUS_OK;
    Scalars s;
    CK(cudaMemcpyAsync(&s, c->sc, sizeof s, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    long long head = s.ring_head, tail = c->ring_tail;
    if (head - tail > c->P.ring_cap) tail = head - c->P.ring_cap;
    long long avail = head - tail;
    if (out && cap > 0) {
        long long nrec = avail < cap ? avail : cap;
        const size_t rec = (size_t)c->P.n_probes * IC_NPROBE_REC;
        for (long long q = 0; q < nrec; ++q) {
            long long slot = (tail + q) % c->P.ring_cap;
            CK(cudaMemcpyAsync(out + q * rec, c->ring + slot * rec, rec * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        }
        CK(cudaStreamSynchronize(c->stream));
        c->ring_tail = tail + nrec;
        if (n_written) *n_written = (int)nrec;
    }
    if (s.status) return status_fail(s.status);
    return ICARUS_OK;
}

int icarus_destroy(icarus_ctx *c)
{
    if (!c) return ICARUS_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graph(c);
    dfree_all(c);
    if (c->hstage) cudaFreeHost(c->hstage);
    if (c->hstatus) cudaFreeHost(c->hstatus);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return ICARUS_OK;
}

int icarus_get_state(icarus_ctx *c, double *U, double *t)
{
    if (!c || !U) return fail(ICARUS_EINVAL, "NULL argument");
    const Params &P = c->P;
    const size_t n = NV * (size_t)P.n1 * P.n2 * P.n3;
    c->ops.pack(P, c->U, c->stage_buf, c->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(U, c->stage_buf, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    Scalars s;
    CK(cudaMemcpyAsync(&s, c->sc, sizeof s, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (t) *t = s.t;
    if (s.status) return status_fail(s.status);
    return ICARUS_OK;
}

int icarus_set_state(icarus_ctx *c, const double *U, double t)
{
    if (!c || !U) return fail(ICARUS_EINVAL, "NULL argument");
    const Params &P = c->P;
    const size_t n = NV * (size_t)P.n1 * P.n2 * P.n3;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpyAsync(c->stage_buf, U, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    c->ops.unpack(P, c->U, c->stage_buf, c->stream);
    c->ops.prims(P, c->U, c->W, c->stream);
    Scalars s;
    CK(cudaMemcpyAsync(&s, c->sc, sizeof s, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    s.t = t;
    s.status = 0;
    s.done = 0;
    if (c->hstatus) *(volatile int *)c->hstatus = 0;
    CK(cudaMemcpyAsync(c->sc, &s, sizeof s, cudaMemcpyHostToDevice, c->stream));
    if (c->opts.tracer) c->ops.tracer_set(P, nullptr, c->U, c->T, c->C, c->stream);   // keep rho c, c = rho c / rho
    c->have_state = true;
    if (c->grid.bc[0] == ICARUS_BC_DRIVEN && !c->have_boundary) {
        CK(cudaStreamSynchronize(c->stream));
        return ICARUS_OK;   // dt is computed once the maps arrive
    }
    return first_dt(c);
}

int icarus_set_psi(icarus_ctx *c, const double *p)
{
    if (!c || !p) return fail(ICARUS_EINVAL, "NULL argument");
    if (c->P.divb != ICARUS_DIVB_GLM) return fail(ICARUS_EINVAL, "the context carries no GLM psi (divb != GLM)");
    const size_t n = (size_t)c->P.n1 * c->P.n2 * c->P.n3;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpyAsync(c->stage_buf, p, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    c->ops.psi_copy(c->P, c->Psi, c->stage_buf, 1, c->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    return ICARUS_OK;
}

int icarus_get_psi(icarus_ctx *c, double *p)
{
    if (!c || !p) return fail(ICARUS_EINVAL, "NULL argument");
    if (c->P.divb != ICARUS_DIVB_GLM) return fail(ICARUS_EINVAL, "the context carries no GLM psi (divb != GLM)");
    const size_t n = (size_t)c->P.n1 * c->P.n2 * c->P.n3;
    c->ops.psi_copy(c->P, c->Psi, c->stage_buf, 0, c->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(p, c->stage_buf, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ICARUS_OK;
}

int icarus_set_tracer(icarus_ctx *c, const double *cin)
{
    if (!c || !cin) return fail(ICARUS_EINVAL, "NULL argument");
    if (!c->opts.tracer) return fail(ICARUS_EINVAL, "the context carries no tracer (options.tracer = 0)");
    if (!c->have_state) return fail(ICARUS_ESTATE, "no state yet: set_state or set_boundary first");
    const size_t n = (size_t)c->P.n1 * c->P.n2 * c->P.n3;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpyAsync(c->stage_buf, cin, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    c->ops.tracer_set(c->P, c->stage_buf, c->U, c->T, c->C, c->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    return ICARUS_OK;
}

int icarus_get_tracer(icarus_ctx *c, double *cout)
{
    if (!c || !cout) return fail(ICARUS_EINVAL, "NULL argument");
    if (!c->opts.tracer) return fail(ICARUS_EINVAL, "the context carries no tracer (options.tracer = 0)");
    if (!c->have_state) return fail(ICARUS_ESTATE, "no state yet: set_state or set_boundary first");
    const size_t n = (size_t)c->P.n1 * c->P.n2 * c->P.n3;
    c->ops.tracer_get(c->P, c->T, c->U, c->stage_buf, c->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(cout, c->stage_buf, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ICARUS_OK;
}

int icarus_copy_state(icarus_ctx *c, double *U_dev)
{
    if (!c || !U_dev) return fail(ICARUS_EINVAL, "NULL argument");
    c->ops.pack(c->P, c->U, U_dev, c->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    return ICARUS_OK;
}

int icarus_set_stop_time(icarus_ctx *c, double t_stop)
{
    if (!c) return fail(ICARUS_EINVAL, "NULL context");
    Scalars s;
    CK(cudaMemcpyAsync(&s, c->sc, sizeof s, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    s.t_stop = t_stop;
    CK(cudaMemcpyAsync(c->sc, &s, sizeof s, cudaMemcpyHostToDevice, c->stream));
    if (c->have_state && (c->grid.bc[0] != ICARUS_BC_DRIVEN || c->have_boundary)) return first_dt(c);
    CK(cudaStreamSynchronize(c->stream));
    return ICARUS_OK;
}

int icarus_time(icarus_ctx *c, double *t, double *dt)
{
    if (!c) return fail(ICARUS_EINVAL, "NULL context");
    Scalars s;
    CK(cudaMemcpyAsync(&s, c->sc, sizeof s, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (t) *t = s.t;
    if (dt) *dt = s.dt;
    return ICARUS_OK;
}

int icarus_math_check(int n, const double *x, double *y)
{
    if (n < 1 || n > (1 << 24) || !x || !y) return fail(ICARUS_EINVAL, "n in [1, 2^24], x and y host arrays");
    double *d = nullptr;
    CK(cudaMalloc(&d, (size_t)5 * n * sizeof(double)));
    cudaError_t e = cudaMemcpy(d, x, (size_t)n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_math_check<<<(n + 255) / 256, 256>>>(d, d + n, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(y, d + n, (size_t)4 * n * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(ICARUS_ECUDA, "math check: %s", cudaGetErrorString(e));
    return ICARUS_OK;
}

int icarus_status(icarus_ctx *c, long long *floor_hits)
{
    if (!c) return fail(ICARUS_EINVAL, "NULL context");
    Scalars s;
    CK(cudaMemcpyAsync(&s, c->sc, sizeof s, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (floor_hits) *floor_hits = (long long)s.floor_hits;
    if (s.status) return status_fail(s.status);
    return ICARUS_OK;
}

int icarus_scales(icarus_ctx *c, double *s)
{
    if (!c || !s) return fail(ICARUS_EINVAL, "NULL argument");
    s[0] = c->t0; s[1] = c->p0; s[2] = c->b0; s[3] = c->omega_code; s[4] = c->gm_code;
    return ICARUS_OK;
}

int icarus_launches_per_step(icarus_ctx *c)
{
    if (!c) return fail(ICARUS_EINVAL, "NULL context");
    return count_launches(c);
}

void *icarus_get_stream(icarus_ctx *c) { return c ? (void *)c->stream : nullptr; }

int icarus_time_kernels(icarus_ctx *c, int n_steps, double *ms)
{
    if (!c || !ms || n_steps < 1) return fail(ICARUS_EINVAL, "bad argument");
    if (!c->have_state) return fail(ICARUS_ESTATE, "no state");
    const int NCLS = ICARUS_KERNEL_CLASSES;
    const bool fused = use_fused_stage(c), rf = use_update_rf(c);
    cudaEvent_t ev[2];
    CK(cudaEventCreate(&ev[0]));
    CK(cudaEventCreate(&ev[1]));
    double acc[NCLS] = {0};
    int cnt[NCLS] = {0};
    const Params &P = c->P;
    cudaStream_t s = c->stream;
    auto timed = [&](int cls, auto &&fn) -> int {
        CK(cudaEventRecord(ev[0], s));
        fn();
        CK(cudaEventRecord(ev[1], s));
        CK(cudaEventSynchronize(ev[1]));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, ev[0], ev[1]));
        acc[cls] += t;
        cnt[cls] += 1;
        return 0;
    };
    int rc = 0;
    for (int q = 0; q < n_steps && !rc; ++q) {
        for (int stage = 1; stage <= 2 && !rc; ++stage) {
            void *Us = stage == 1 ? c->U : c->U1, *Ws = stage == 1 ? c->W : c->W1;
            void *Uo = stage == 1 ? c->U1 : c->U, *Wo = stage == 1 ? c->W1 : c->W;
            rc |= timed(0, [&] { c->ops.fill_ghosts(P, Us, Ws, stage, s); });
            if (fused) {
                rc |= timed(7 + stage, [&] { c->ops.fused_stage(P, stage, Us, Ws, Uo, Wo, s); });
                continue;
            }
            if (!rf) rc |= timed(1, [&] { c->ops.flux_dir(P, 0, Ws, c->F1, s); });
            rc |= timed(2, [&] { c->ops.flux_dir(P, 1, Ws, c->F2, s); });
            rc |= timed(3, [&] { c->ops.flux_dir(P, 2, Ws, c->F3, s); });
            if (P.divb == 1 || P.divb == 3) rc |= timed(4, [&] { c->ops.divb(P, Ws, c->divB, s); });
            if (rf) rc |= timed(4 + stage, [&] { c->ops.update_rf(P, stage, Us, Ws, Uo, Wo, c->F2, c->F3, c->divB, s); });
            else rc |= timed(4 + stage, [&] { c->ops.update(P, stage, Us, Ws, Uo, Wo, c->F1, c->F2, c->F3, c->divB, s); });
        }
        if (P.n_probes > 0) rc |= timed(7, [&] { c->ops.probe(P, c->W, s); });
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc) return rc;
    CK(cudaGetLastError());
    for (int k = 0; k < NCLS; ++k) ms[k] = cnt[k] ? acc[k] / cnt[k] : 0.0;
    return ICARUS_OK;
}

}  // extern "C"
