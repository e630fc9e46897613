// icarus_noalloc.cu -- allocation-free variant of the CFL time-step reduction.
//
// Some callers cannot allocate device memory at the point where they need a time step: code that
// runs under another framework's fixed memory budget or pool, real-time drivers that forbid
// allocation after start-up, or embedders whose only device memory is the buffers they already
// own. icarus_cfl_dt_noalloc serves them: the caller passes its conserved state and a place for
// the result, and the per-block partial maxima plus the last-block counter of the reduction live
// in one file-scope device array of fixed size (ICARUS_NOALLOC_MAX_CELLS / 256 partials, 128 KiB),
// which every GPU that loads the library keeps until the process exits.
#include <mutex>

#include "../../include/icarus.h"
#include "icarus_kernels.cuh"

using namespace icarus;

namespace {

constexpr int NA_BLOCK = 256;
constexpr long long NA_MAX_BLOCKS = ICARUS_NOALLOC_MAX_CELLS / NA_BLOCK;
constexpr int NA_HEADER = 32;   // first 256 bytes: the last-block counter and the non-finite flag
                                // (two unsigned ints), then padding

// scratch shared by every call on a device: [counter | pad][partial maxima]
static __device__ __align__(256) double g_cfl_scratch[NA_HEADER + NA_MAX_BLOCKS];

struct NaGrid {
    int n1, n2, n3, geom, stretch, band_refine;
    double x1min, x1max, x2min, d2, x3min, d3, band_lo, band_hi, gamma, cfl;
};

// radial edge i: the refined band's edges when there is one, else geometric (stretched sphere) or
// uniform spacing -- the edges the context builds for its metric tables
__device__ double na_edge1(const NaGrid &g, int i)
{
    const bool lg = g.geom == ICARUS_GEOM_SPHERICAL && g.stretch;
    if (g.band_refine > 1) return band_edge_at(g.n1, g.x1min, g.x1max, g.band_lo, g.band_hi, g.band_refine, lg, i);
    if (lg) return g.x1min * pow(g.x1max / g.x1min, (double)i / g.n1);
    return g.x1min + i * ((g.x1max - g.x1min) / g.n1);
}

// one thread per interior cell: primitives from the conserved state, the cell's signal speed
// sum_d (|v_d| + c_f,d) / dx_d, block max, then the last block turns the maximum into dt
__global__ void __launch_bounds__(NA_BLOCK) k_cfl_noalloc(NaGrid g, const double *__restrict__ U, double *dt_out,
                                                          double *scratch)
{
    unsigned int *done = reinterpret_cast<unsigned int *>(scratch);
    unsigned int *nonfinite = done + 1;
    double *partial = scratch + NA_HEADER;
    const long long N = (long long)g.n1 * g.n2 * g.n3;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (tid < N) {
        const int i = (int)(tid % g.n1);
        const long long r_ = tid / g.n1;
        const int j = (int)(r_ % g.n2);
        double u[NV], w[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = U[v * N + tid];
        cons2prim<double>(u, w, g.gamma - 1.0);
        const double rm = na_edge1(g, i), rp = na_edge1(g, i + 1);
        double w1 = rp - rm, w2 = g.d2, w3 = g.d3;
        if (g.geom == ICARUS_GEOM_SPHERICAL) {
            const double rc = 0.5 * (rm + rp);
            const double th = 0.5 * ((g.x2min + j * g.d2) + (g.x2min + (j + 1) * g.d2));
            w2 = rc * g.d2;
            w3 = rc * sin(th) * g.d3;
        }
        const double irho = 1.0 / w[0];
        s = (fabs(w[1]) + fast_speed<double>(w, irho, 0, g.gamma)) / w1
          + (fabs(w[2]) + fast_speed<double>(w, irho, 1, g.gamma)) / w2
          + (fabs(w[3]) + fast_speed<double>(w, irho, 2, g.gamma)) / w3;
    }
    // fmax in the reduction would drop a NaN: a non-finite speed is flagged on its own
    const int bad = __syncthreads_or(!isfinite(s));
    s = block_max(s);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        if (bad) atomicOr(nonfinite, 1u);
        partial[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) v = fmax(v, ((volatile double *)partial)[b]);
    v = block_max(v);
    if (threadIdx.x == 0) {
        const bool any_bad = ((volatile unsigned int *)nonfinite)[0] != 0u;
        *dt_out = any_bad ? -1.0 : (v > 0.0 ? g.cfl / v : 0.0);
        *done = 0;
        *nonfinite = 0;
    }
}

std::mutex g_setup_mu;
double *g_scratch_dev[256];
bool g_scratch_ready[256];

int na_fail(int code, const char *msg) { return icarus::report_error(code, msg); }

}  // namespace

extern "C" int icarus_cfl_dt_noalloc(const icarus_grid *grid, double gamma, double cfl, const double *U, double *dt,
                                     void *stream)
{
    if (!grid || !U || !dt) return na_fail(ICARUS_EINVAL, "NULL argument");
    // the grids icarus_init accepts, no others (message from the shared check)
    if (check_grid(grid) != ICARUS_OK) return ICARUS_EINVAL;
    const long long N = (long long)grid->n1 * grid->n2 * grid->n3;
    if (N > ICARUS_NOALLOC_MAX_CELLS)
        return na_fail(ICARUS_EINVAL, "grid has more cells than ICARUS_NOALLOC_MAX_CELLS (4194304); use icarus_set_state + icarus_time");
    if (!(gamma > 1.0) || !(cfl > 0.0 && cfl <= 1.0)) return na_fail(ICARUS_EINVAL, "need gamma > 1 and cfl in (0, 1]");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return na_fail(ICARUS_ECUDA, "no current CUDA device");
    {
        // once per device, with that device current: the device address of the scratch array
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_scratch_ready[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_cfl_scratch);
            if (e != cudaSuccess || !p) return na_fail(ICARUS_ECUDA, cudaGetErrorString(e));
            g_scratch_dev[dev] = (double *)p;
            g_scratch_ready[dev] = true;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *scratch = g_scratch_dev[dev];
    // counter and flag must start at zero even if an earlier call on this device was interrupted
    if (cudaMemsetAsync(scratch, 0, 2 * sizeof(unsigned int), s) != cudaSuccess)
        return na_fail(ICARUS_ECUDA, "memset of the counter failed");
    NaGrid g;
    g.n1 = grid->n1; g.n2 = grid->n2; g.n3 = grid->n3;
    g.geom = grid->geometry; g.stretch = grid->stretch;
    g.x1min = grid->x1min; g.x1max = grid->x1max;
    g.x2min = grid->x2min; g.d2 = (grid->x2max - grid->x2min) / grid->n2;
    g.x3min = grid->x3min; g.d3 = (grid->x3max - grid->x3min) / grid->n3;
    g.band_refine = grid->band_refine; g.band_lo = grid->band_lo; g.band_hi = grid->band_hi;
    g.gamma = gamma; g.cfl = cfl;
    const unsigned int blocks = (unsigned int)((N + NA_BLOCK - 1) / NA_BLOCK);
    k_cfl_noalloc<<<blocks, NA_BLOCK, 0, s>>>(g, U, dt, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(ICARUS_ECUDA, cudaGetErrorString(e));
    return ICARUS_OK;
}
