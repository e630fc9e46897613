// icarus_batch.cuh -- batched ensemble: every member's whole time step in ONE persistent,
// cooperatively launched kernel. Members have their own grids (uneven sizes), boundary drivers,
// CMEs, dt and t. Work is cut into (member, tile) items per phase; the blocks stride over the
// items of a phase, then meet at a grid barrier (bounded spin: a barrier that does not complete
// within the limit sets an error word and the kernel returns). Phases per step:
//   stage s = 1, 2: ghost r | ghost theta | ghost phi | fluxes r+theta+phi | div B | update
//   then: per-member dt / t | probes
// The tile shape of the flux phases is chosen per member from a candidate set (autotuned per grid
// shape on the host); all per-cell and per-face arithmetic is the single-solver code.
#pragma once
#include "icarus_kernels.cuh"

namespace icarus {

// work-item tables: the persistent kernel uses the first BPH_NP (fluxes of all directions in one
// phase); the per-phase form takes the fluxes direction by direction (BPH_FR, BPH_FT, BPH_FP)
enum { BPH_BND1 = 0, BPH_BND2, BPH_BND3, BPH_FLUX, BPH_DIVB, BPH_UPD, BPH_PROBE, BPH_NP,
       BPH_FR = BPH_NP, BPH_FT, BPH_FP, BPH_N };
constexpr int BATCH_THREADS = 256;
// flux tile candidates (BX x BY = 256 threads): r faces (128x2, 64x4, 32x8); theta / phi faces
// (16x16, 32x8)
constexpr int NCFG_R = 3, NCFG_T = 2;

struct Member {
    Params P;
    void *U, *U1, *W, *W1, *F1, *F2, *F3, *divB;
    int cfg_r, cfg_t;
    int tr[3], tt[3], tp[3];           // tiles along the three launch axes (r, theta, phi fluxes)
    long long items_r, items_t, items_p;
};

struct BarrierState {
    unsigned int count, gen;           // reset before every launch
    unsigned int pad[2];
    int err;                           // sticky: 1 = a barrier wait gave up
};

struct BatchArgs {
    const Member *m;
    const long long *off;              // [BPH_N][n + 1] prefix sums of work items
    int n;
    BarrierState *bar;
    long long spin_limit;              // clock64 ticks a barrier may wait
};

__device__ __forceinline__ int find_member(const long long *off, int n, long long it)
{
    int lo = 0, hi = n;                // largest m with off[m] <= it
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= it) lo = mid; else hi = mid;
    }
    return lo;
}

// grid-wide barrier for a cooperative launch; false if the wait gave up (error recorded)
__device__ __forceinline__ bool grid_sync(const BatchArgs &A)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = &A.bar->gen;
        const unsigned int g = *vgen;
        __threadfence();
        ok = 1;
        if (atomicAdd(&A.bar->count, 1u) == gridDim.x - 1) {
            atomicExch(&A.bar->count, 0u);
            __threadfence();
            atomicAdd(&A.bar->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g) {
                if (clock64() - t0 > A.spin_limit) { atomicOr(&A.bar->err, 1); ok = 0; break; }
                __nanosleep(100);
            }
        }
        __threadfence();
        if (*(volatile int *)&A.bar->err) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

// self-test of the bounded barrier: every block but `absent` (-1: none) meets at one barrier; a
// block that never arrives makes the others give up after spin_limit clock ticks and record it
static __global__ void k_barrier_selftest(BatchArgs A, int absent)
{
    if ((int)blockIdx.x == absent) return;
    grid_sync(A);
}

template <int D, int BX, int BY, typename TW>
__device__ __forceinline__ void flux_item(const Member &M, const TW *W, TW *F, long long local, const int *nt,
                                          TW *smem)
{
    // tile counts per member stay far below 2^32: 32-bit divisions (a 64-bit one is a long
    // software sequence, paid by every thread of every tile)
    const unsigned int l32 = (unsigned int)local, n0 = (unsigned int)nt[0], n1 = (unsigned int)nt[1];
    const unsigned int r_ = l32 / n0;
    const int bx = (int)(l32 - r_ * n0);
    const int by = (int)(r_ % n1), bz = (int)(r_ / n1);
    flux_tile<D, BX, BY, TW>(M.P, W, F, bx, by, bz, threadIdx.x % BX, threadIdx.x / BX, smem, smem + NV * BX * BY);
}

// two resident blocks per SM at least (three when the arithmetic is single precision)
// the item index only grows inside a phase loop, so the member index is found by advancing
__device__ __forceinline__ int next_member(const long long *off, int n, long long it, int m)
{
    while (m + 1 < n && off[m + 1] <= it) ++m;
    return m;
}

// the persistent kernel's copy of the current member's descriptor in shared memory, refreshed when
// the block's item moves to another member (items are block-uniform, so is m)
__device__ __forceinline__ const Member &member_cached(const BatchArgs &A, int m, Member &sm, int &cached)
{
    if (m != cached) {
        __syncthreads();                  // nobody still reads the previous member
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(A.m + m);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(&sm);
        for (int q = threadIdx.x; q < (int)(sizeof(Member) / 8); q += blockDim.x) dst[q] = src[q];
        __syncthreads();
        cached = m;
    }
    return sm;
}

template <typename TS, typename TW>
__global__ void __launch_bounds__(BATCH_THREADS, sizeof(TW) == 4 ? 4 : 2) k_batch_step(BatchArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TW *smem = reinterpret_cast<TW *>(smem_raw);
    // work-item prefix sums of all phases, kept in shared memory after the flux tiles
    long long *soff = reinterpret_cast<long long *>(smem_raw + 2 * NV * BATCH_THREADS * sizeof(TW));
    for (int q = threadIdx.x; q < BPH_NP * (A.n + 1); q += blockDim.x) soff[q] = A.off[q];
    __shared__ Member sm_member;
    int cached = -1;
    __syncthreads();
    const int tid = threadIdx.x;
    for (int stage = 1; stage <= 2; ++stage) {
        // ---- ghost fill, r
        {
            const long long *off = soff + (long long)BPH_BND1 * (A.n + 1);
            int m = 0;
            for (long long it = blockIdx.x; it < off[A.n]; it += gridDim.x) {
                m = next_member(off, A.n, it, m);
                const Member &M = member_cached(A, m, sm_member, cached);
                const long long c = (it - off[m]) * BATCH_THREADS + tid;
                if (c < (long long)M.P.n2 * M.P.n3)
                    bnd1_col<TS, TW>(M.P, (TS *)(stage == 1 ? M.U : M.U1), (TW *)(stage == 1 ? M.W : M.W1), stage,
                                     (int)((unsigned int)c % (unsigned int)M.P.n2), (int)((unsigned int)c / (unsigned int)M.P.n2));
            }
        }
        if (!grid_sync(A)) return;
        // ---- ghost fill, theta (every r incl. ghosts, interior phi)
        {
            const long long *off = soff + (long long)BPH_BND2 * (A.n + 1);
            int m = 0;
            for (long long it = blockIdx.x; it < off[A.n]; it += gridDim.x) {
                m = next_member(off, A.n, it, m);
                const Member &M = member_cached(A, m, sm_member, cached);
                const long long c = (it - off[m]) * BATCH_THREADS + tid;
                if (c < (long long)M.P.p1 * M.P.n3)
                    bnd23_cell<1, TS, TW>(M.P, (TS *)(stage == 1 ? M.U : M.U1), (TW *)(stage == 1 ? M.W : M.W1),
                                          (int)((unsigned int)c % (unsigned int)M.P.p1), (int)((unsigned int)c / (unsigned int)M.P.p1));
            }
        }
        if (!grid_sync(A)) return;
        // ---- ghost fill, phi (everything)
        {
            const long long *off = soff + (long long)BPH_BND3 * (A.n + 1);
            int m = 0;
            for (long long it = blockIdx.x; it < off[A.n]; it += gridDim.x) {
                m = next_member(off, A.n, it, m);
                const Member &M = member_cached(A, m, sm_member, cached);
                const long long c = (it - off[m]) * BATCH_THREADS + tid;
                if (c < (long long)M.P.p1 * M.P.p2)
                    bnd23_cell<2, TS, TW>(M.P, (TS *)(stage == 1 ? M.U : M.U1), (TW *)(stage == 1 ? M.W : M.W1),
                                          (int)((unsigned int)c % (unsigned int)M.P.p1), (int)((unsigned int)c / (unsigned int)M.P.p1));
            }
        }
        if (!grid_sync(A)) return;
        // ---- face fluxes, all three directions
        {
            const long long *off = soff + (long long)BPH_FLUX * (A.n + 1);
            int m = 0;
            for (long long it = blockIdx.x; it < off[A.n]; it += gridDim.x) {
                m = next_member(off, A.n, it, m);
                const Member &M = member_cached(A, m, sm_member, cached);
                long long local = it - off[m];
                const TW *W = (const TW *)(stage == 1 ? M.W : M.W1);
                if (local < M.items_r) {
                    if (M.cfg_r == 0) flux_item<0, 128, 2, TW>(M, W, (TW *)M.F1, local, M.tr, smem);
                    else if (M.cfg_r == 1) flux_item<0, 64, 4, TW>(M, W, (TW *)M.F1, local, M.tr, smem);
                    else flux_item<0, 32, 8, TW>(M, W, (TW *)M.F1, local, M.tr, smem);
                } else if ((local -= M.items_r) < M.items_t) {
                    if (M.cfg_t == 0) flux_item<1, 16, 16, TW>(M, W, (TW *)M.F2, local, M.tt, smem);
                    else flux_item<1, 32, 8, TW>(M, W, (TW *)M.F2, local, M.tt, smem);
                } else {
                    local -= M.items_t;
                    if (M.cfg_t == 0) flux_item<2, 16, 16, TW>(M, W, (TW *)M.F3, local, M.tp, smem);
                    else flux_item<2, 32, 8, TW>(M, W, (TW *)M.F3, local, M.tp, smem);
                }
                __syncthreads();           // the next item reuses the shared tile
            }
        }
        if (!grid_sync(A)) return;
        // ---- div B
        {
            const long long *off = soff + (long long)BPH_DIVB * (A.n + 1);
            int m = 0;
            for (long long it = blockIdx.x; it < off[A.n]; it += gridDim.x) {
                m = next_member(off, A.n, it, m);
                const Member &M = member_cached(A, m, sm_member, cached);
                const long long c = (it - off[m]) * BATCH_THREADS + tid;
                if (c < (long long)(M.P.n1 + 2) * (M.P.n2 + 2) * (M.P.n3 + 2))
                    divb_cell<TW>(M.P, (const TW *)(stage == 1 ? M.W : M.W1), (TW *)M.divB, c);
            }
        }
        if (!grid_sync(A)) return;
        // ---- update (stage 2 also reduces each member's CFL speed)
        {
            const long long *off = soff + (long long)BPH_UPD * (A.n + 1);
            int m = 0;
            for (long long it = blockIdx.x; it < off[A.n]; it += gridDim.x) {
                m = next_member(off, A.n, it, m);
                const Member &M = member_cached(A, m, sm_member, cached);
                const long long c = (it - off[m]) * BATCH_THREADS + tid;
                const bool valid = c < (long long)M.P.n1 * M.P.n2 * M.P.n3;
                TW wo[NV];
                if (valid) {
                    if (stage == 1)
                        update_cell<1, TS, TW>(M.P, (const TS *)M.U, (const TW *)M.W, (TS *)M.U1, (TW *)M.W1,
                                               (const TW *)M.F1, (const TW *)M.F2, (const TW *)M.F3,
                                               (const TW *)M.divB, c, wo);
                    else
                        update_cell<2, TS, TW>(M.P, (const TS *)M.U1, (const TW *)M.W1, (TS *)M.U, (TW *)M.W,
                                               (const TW *)M.F1, (const TW *)M.F2, (const TW *)M.F3,
                                               (const TW *)M.divB, c, wo);
                }
                if (stage == 2) {
                    const unsigned int c32 = (unsigned int)c, n1u = (unsigned int)M.P.n1;
                    const int ci = valid ? (int)(c32 % n1u) : 0, cj = valid ? (int)((c32 / n1u) % (unsigned int)M.P.n2) : 0;
                    const double smax = cfl_block_speed<TW>(M.P, wo, ci + NG, cj + NG, valid);
                    if (tid == 0) atomicMax(&M.P.sc->smax_bits, (unsigned long long)__double_as_longlong(smax));
                }
            }
        }
        if (!grid_sync(A)) return;
    }
    // ---- per-member dt and t (the arithmetic of the single solver's last-block finalisation)
    for (int m = blockIdx.x * blockDim.x + tid; m < A.n; m += gridDim.x * blockDim.x) {
        Scalars *sc = A.m[m].P.sc;
        const double v = __longlong_as_double((long long)sc->smax_bits);
        const double t = __dadd_rn(sc->t, sc->dt);
        double dt = sc->cfl / v;
        if (sc->t_stop > 0.0) dt = fmin(dt, fmax(__dsub_rn(sc->t_stop, t), 0.0));
        if (!(v > 0.0)) dt = 0.0;
        sc->t = t;
        sc->dt = dt;
        sc->smax_bits = 0ull;
    }
    if (!grid_sync(A)) return;
    // ---- probes: one item per member that has them
    {
        const long long *off = soff + (long long)BPH_PROBE * (A.n + 1);
        for (long long it = blockIdx.x; it < off[A.n]; it += gridDim.x) {
            const int m = find_member(off, A.n, it);
            const Member &M = A.m[m];
            const long long head = M.P.sc->ring_head;
            __syncthreads();
            for (int p = tid; p < M.P.n_probes; p += blockDim.x) probe_one<TW>(M.P, (const TW *)M.W, p, head);
            __syncthreads();
            if (tid == 0) M.P.sc->ring_head = head + 1;
        }
    }
}

// the block's member descriptor copied into shared memory: every thread then reads its fields
// with broadcast shared loads (the descriptor in global memory would be re-read after each global
// store, since the compiler cannot rule out that the store changed it)
__device__ __forceinline__ const Member &stage_member(const BatchArgs &A, int m, Member &sm)
{
    static_assert(sizeof(Member) % 8 == 0, "Member is copied in 8-byte words");
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(A.m + m);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(&sm);
    for (int q = threadIdx.x; q < (int)(sizeof(Member) / 8); q += blockDim.x) dst[q] = src[q];
    __syncthreads();
    return sm;
}

// ---- per-phase form: the same phases as separate launches, each over the items of ALL members
// (one item per block), so that every phase keeps its own register budget and occupancy (the
// persistent kernel runs every phase at the budget of the largest one). A stream-ordered launch
// boundary replaces each grid barrier; a step is 14 launches whatever the number of members.
template <typename TS, typename TW>
__global__ void __launch_bounds__(BATCH_THREADS) k_bp_ghost(BatchArgs A, int phase, int stage)
{
    const long long *off = A.off + (long long)phase * (A.n + 1);
    const long long it = blockIdx.x;
    const int m = find_member(off, A.n, it);
    __shared__ Member sm_member;
    const Member &M = stage_member(A, m, sm_member);
    const long long c = (it - off[m]) * BATCH_THREADS + threadIdx.x;
    TS *U = (TS *)(stage == 1 ? M.U : M.U1);
    TW *W = (TW *)(stage == 1 ? M.W : M.W1);
    const unsigned int c32 = (unsigned int)c;    // below the padded cell count, < 2^31
    if (phase == BPH_BND1) {
        const unsigned int n2 = (unsigned int)M.P.n2;
        if (c < (long long)M.P.n2 * M.P.n3) bnd1_col<TS, TW>(M.P, U, W, stage, (int)(c32 % n2), (int)(c32 / n2));
    } else {
        const unsigned int p1 = (unsigned int)M.P.p1;
        if (phase == BPH_BND2) {
            if (c < (long long)M.P.p1 * M.P.n3) bnd23_cell<1, TS, TW>(M.P, U, W, (int)(c32 % p1), (int)(c32 / p1));
        } else {
            if (c < (long long)M.P.p1 * M.P.p2) bnd23_cell<2, TS, TW>(M.P, U, W, (int)(c32 % p1), (int)(c32 / p1));
        }
    }
}

// the fluxes of one direction D for every member, one tile shape for the whole launch (chosen for
// the ensemble by the autotuner): one code path per launch, as in the single solver's kernels
template <int D, int BX, int BY, typename TW>
__global__ void __launch_bounds__(BATCH_THREADS) k_bp_flux(BatchArgs A, int stage)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TW *smem = reinterpret_cast<TW *>(smem_raw);
    const long long *off = A.off + (long long)(BPH_FR + D) * (A.n + 1);
    const long long it = blockIdx.x;
    const int m = find_member(off, A.n, it);
    __shared__ Member sm_member;
    const Member &M = stage_member(A, m, sm_member);
    const TW *W = (const TW *)(stage == 1 ? M.W : M.W1);
    TW *F = (TW *)(D == 0 ? M.F1 : (D == 1 ? M.F2 : M.F3));
    flux_item<D, BX, BY, TW>(M, W, F, it - off[m], D == 0 ? M.tr : (D == 1 ? M.tt : M.tp), smem);
}

template <int D, int BX, int BY, typename TW>
inline void launch_bp_flux(const BatchArgs &A, long long items, int stage, cudaStream_t s)
{
    if (items) k_bp_flux<D, BX, BY, TW><<<(unsigned)items, BATCH_THREADS, 2 * NV * BX * BY * sizeof(TW), s>>>(A, stage);
}

template <typename TW>
__global__ void __launch_bounds__(BATCH_THREADS) k_bp_divb(BatchArgs A, int stage)
{
    const long long *off = A.off + (long long)BPH_DIVB * (A.n + 1);
    const long long it = blockIdx.x;
    const int m = find_member(off, A.n, it);
    __shared__ Member sm_member;
    const Member &M = stage_member(A, m, sm_member);
    const long long c = (it - off[m]) * BATCH_THREADS + threadIdx.x;
    if (c < (long long)(M.P.n1 + 2) * (M.P.n2 + 2) * (M.P.n3 + 2))
        divb_cell<TW>(M.P, (const TW *)(stage == 1 ? M.W : M.W1), (TW *)M.divB, c);
}

template <int STAGE, typename TS, typename TW>
__device__ __forceinline__ void bp_update_body(const BatchArgs &A)
{
    const long long *off = A.off + (long long)BPH_UPD * (A.n + 1);
    const long long it = blockIdx.x;
    const int m = find_member(off, A.n, it);
    __shared__ Member sm_member;
    const Member &M = stage_member(A, m, sm_member);
    const long long c = (it - off[m]) * BATCH_THREADS + threadIdx.x;
    const bool valid = c < (long long)M.P.n1 * M.P.n2 * M.P.n3;
    TW wo[NV];
    if (valid) {
        if (STAGE == 1)
            update_cell<1, TS, TW>(M.P, (const TS *)M.U, (const TW *)M.W, (TS *)M.U1, (TW *)M.W1, (const TW *)M.F1,
                                   (const TW *)M.F2, (const TW *)M.F3, (const TW *)M.divB, c, wo);
        else
            update_cell<2, TS, TW>(M.P, (const TS *)M.U1, (const TW *)M.W1, (TS *)M.U, (TW *)M.W, (const TW *)M.F1,
                                   (const TW *)M.F2, (const TW *)M.F3, (const TW *)M.divB, c, wo);
    }
    if (STAGE == 2) {
        const unsigned int c32 = (unsigned int)c, n1 = (unsigned int)M.P.n1;
        const int ci = valid ? (int)(c32 % n1) : 0, cj = valid ? (int)((c32 / n1) % (unsigned int)M.P.n2) : 0;
        const double smax = cfl_block_speed<TW>(M.P, wo, ci + NG, cj + NG, valid);
        if (threadIdx.x == 0) atomicMax(&M.P.sc->smax_bits, (unsigned long long)__double_as_longlong(smax));
    }
}

// the update's register budget as in the single solver: the second single-precision stage of the
// mixed form capped at 48 registers (5 blocks per SM), the others uncapped
template <int STAGE, typename TS, typename TW>
__global__ void __launch_bounds__(BATCH_THREADS) k_bp_update(BatchArgs A) { bp_update_body<STAGE, TS, TW>(A); }
template <int STAGE, typename TS, typename TW>
__global__ void __launch_bounds__(BATCH_THREADS, 5) k_bp_update_capped(BatchArgs A) { bp_update_body<STAGE, TS, TW>(A); }

// per-member dt and t after the second stage (the arithmetic of the single solver's finalisation)
static __global__ void k_bp_finish(BatchArgs A)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < A.n; m += gridDim.x * blockDim.x) {
        Scalars *sc = A.m[m].P.sc;
        const double v = __longlong_as_double((long long)sc->smax_bits);
        const double t = __dadd_rn(sc->t, sc->dt);
        double dt = sc->cfl / v;
        if (sc->t_stop > 0.0) dt = fmin(dt, fmax(__dsub_rn(sc->t_stop, t), 0.0));
        if (!(v > 0.0)) dt = 0.0;
        sc->t = t;
        sc->dt = dt;
        sc->smax_bits = 0ull;
    }
}

template <typename TW>
__global__ void __launch_bounds__(BATCH_THREADS) k_bp_probe(BatchArgs A)
{
    const long long *off = A.off + (long long)BPH_PROBE * (A.n + 1);
    const int m = find_member(off, A.n, blockIdx.x);
    __shared__ Member sm_member;
    const Member &M = stage_member(A, m, sm_member);
    const long long head = M.P.sc->ring_head;
    __syncthreads();
    for (int p = threadIdx.x; p < M.P.n_probes; p += blockDim.x) probe_one<TW>(M.P, (const TW *)M.W, p, head);
    __syncthreads();
    if (threadIdx.x == 0) M.P.sc->ring_head = head + 1;
}

// flux kernels of one tile variant, for the autotuner's timed trials
template <int D, int BX, int BY, typename TW>
__global__ void __launch_bounds__(BATCH_THREADS) k_flux_var(Params P, const TW *__restrict__ W, TW *__restrict__ F)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TW *smem = reinterpret_cast<TW *>(smem_raw);
    flux_tile<D, BX, BY, TW>(P, W, F, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x % BX, threadIdx.x / BX, smem,
                             smem + NV * BX * BY);
}

template <int D, int BX, int BY, typename TW>
inline void launch_flux_var(const Params &P, const void *W, void *F, cudaStream_t s)
{
    int nx, ny, nz;
    flux_tiles<D, BX, BY>(P, nx, ny, nz);
    k_flux_var<D, BX, BY, TW><<<dim3(nx, ny, nz), BATCH_THREADS, 2 * NV * BX * BY * sizeof(TW), s>>>(
        P, (const TW *)W, (TW *)F);
}

struct BatchOps {
    cudaError_t (*launch)(const BatchArgs &, int blocks, cudaStream_t);
    // the per-phase form: items[BPH_N] = work items of each phase over all members; the ensemble's
    // flux tile candidates (cfg_r, cfg_t); and one direction's flux launch (autotuner trials)
    cudaError_t (*launch_phases)(const BatchArgs &, const long long *items, int cfg_r, int cfg_t, cudaStream_t);
    cudaError_t (*launch_flux_dir)(const BatchArgs &, int dir, int cfg, long long items, int stage, cudaStream_t);
    int (*blocks_per_sm)(int n_members);
    void (*flux_variant)(const Params &, int dir, int cfg, const void *W, void *F, cudaStream_t);
    size_t tw_size;
};

template <typename TS, typename TW> struct BatchLaunch {
    static size_t smem(int n) { return 2 * NV * BATCH_THREADS * sizeof(TW) + sizeof(long long) * BPH_NP * (n + 1); }
    static cudaError_t launch(const BatchArgs &A, int blocks, cudaStream_t s)
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(blocks);
        cfg.blockDim = dim3(BATCH_THREADS);
        cfg.dynamicSmemBytes = smem(A.n);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_batch_step<TS, TW>, A);
    }
    // the fluxes of direction dir with tile candidate cfg (codes as in Member::cfg_r / cfg_t)
    static cudaError_t launch_flux_dir(const BatchArgs &A, int dir, int cfg, long long items, int stage, cudaStream_t s)
    {
        if (dir == 0) {
            if (cfg == 0) launch_bp_flux<0, 128, 2, TW>(A, items, stage, s);
            else if (cfg == 1) launch_bp_flux<0, 64, 4, TW>(A, items, stage, s);
            else launch_bp_flux<0, 32, 8, TW>(A, items, stage, s);
        } else if (dir == 1) {
            if (cfg == 0) launch_bp_flux<1, 16, 16, TW>(A, items, stage, s);
            else launch_bp_flux<1, 32, 8, TW>(A, items, stage, s);
        } else {
            if (cfg == 0) launch_bp_flux<2, 16, 16, TW>(A, items, stage, s);
            else launch_bp_flux<2, 32, 8, TW>(A, items, stage, s);
        }
        return cudaGetLastError();
    }
    static cudaError_t launch_phases(const BatchArgs &A, const long long *items, int cfg_r, int cfg_t, cudaStream_t s)
    {
        constexpr bool capped2 = sizeof(TS) == 8 && sizeof(TW) == 4;   // mixed form, as in the single solver
        for (int stage = 1; stage <= 2; ++stage) {
            for (int ph = BPH_BND1; ph <= BPH_BND3; ++ph)
                if (items[ph]) k_bp_ghost<TS, TW><<<(unsigned)items[ph], BATCH_THREADS, 0, s>>>(A, ph, stage);
            for (int d = 0; d < 3; ++d) launch_flux_dir(A, d, d == 0 ? cfg_r : cfg_t, items[BPH_FR + d], stage, s);
            if (items[BPH_DIVB]) k_bp_divb<TW><<<(unsigned)items[BPH_DIVB], BATCH_THREADS, 0, s>>>(A, stage);
            if (items[BPH_UPD]) {
                if (stage == 1) k_bp_update<1, TS, TW><<<(unsigned)items[BPH_UPD], BATCH_THREADS, 0, s>>>(A);
                else if constexpr (capped2) k_bp_update_capped<2, TS, TW><<<(unsigned)items[BPH_UPD], BATCH_THREADS, 0, s>>>(A);
                else k_bp_update<2, TS, TW><<<(unsigned)items[BPH_UPD], BATCH_THREADS, 0, s>>>(A);
            }
        }
        k_bp_finish<<<(A.n + 127) / 128, 128, 0, s>>>(A);
        if (items[BPH_PROBE]) k_bp_probe<TW><<<(unsigned)items[BPH_PROBE], BATCH_THREADS, 0, s>>>(A);
        return cudaGetLastError();
    }
    static int blocks_per_sm(int n)
    {
        int nb = 0;
        const size_t sm = smem(n);
        if (sm > 48 * 1024 &&
            cudaFuncSetAttribute(k_batch_step<TS, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
            return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_step<TS, TW>, BATCH_THREADS, sm) != cudaSuccess)
            return 0;
        return nb;
    }
    static void flux_variant(const Params &P, int dir, int cfg, const void *W, void *F, cudaStream_t s)
    {
        if (dir == 0) {
            if (cfg == 0) launch_flux_var<0, 128, 2, TW>(P, W, F, s);
            else if (cfg == 1) launch_flux_var<0, 64, 4, TW>(P, W, F, s);
            else launch_flux_var<0, 32, 8, TW>(P, W, F, s);
        } else if (dir == 1) {
            if (cfg == 0) launch_flux_var<1, 16, 16, TW>(P, W, F, s);
            else launch_flux_var<1, 32, 8, TW>(P, W, F, s);
        } else {
            if (cfg == 0) launch_flux_var<2, 16, 16, TW>(P, W, F, s);
            else launch_flux_var<2, 32, 8, TW>(P, W, F, s);
        }
    }
    static BatchOps make()
    {
        BatchOps o;
        o.launch = launch;
        o.launch_phases = launch_phases;
        o.launch_flux_dir = launch_flux_dir;
        o.blocks_per_sm = blocks_per_sm;
        o.flux_variant = flux_variant;
        o.tw_size = sizeof(TW);
        return o;
    }
};

BatchOps batch_ops_fp64();
BatchOps batch_ops_fp32();
BatchOps batch_ops_mixed();

}  // namespace icarus
