// closure.cu -- learned closure for a coarse solve: a 4-layer 3-D convolutional network
// (8 -> 32 -> 32 -> 32 -> 8 channels, 3x3x3 kernels, ReLU between layers, phi circular and
// r / theta replicate padding) that predicts the correction of a coarse state towards the
// restricted fine solution; trained on the GPU by the kernels below.
//
// Every convolution runs on the tensor cores as an implicit GEMM with BF16 operands and FP32
// accumulation: the forward (rows = voxels, K = 27 taps x C_in) and the data gradient (the same
// convolution over the padded grid with the transposed, tap-reversed weights, rows = padded
// voxels, K = 27 x C_out) on the 5th-generation tensor cores (tcgen05.mma, accumulators in tensor
// memory, operands brought into shared memory by the tensor memory accelerator); the weight
// gradient on the same tensor cores (rows = the three r shifts x C_out, columns = the nine
// (theta, phi) lines x C_in, K = padded positions split over blocks, operands transposed into
// shared memory with movmatrix, blocks' partial sums reduced by a second kernel). Activations are stored
// channels-last on a grid padded by one ghost layer; a pad kernel fills the ghosts (replicate /
// circular) and a fold kernel adds ghost gradients back to the cells they copy (the adjoint).
// Channel counts are padded to multiples of 16 (layer 0 input 8 -> 16 zero channels, layer 3
// output 8 -> 16 with zero weights); the padding never carries a gradient.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "icarus_ctx.h"
#include "icarus_kernels.cuh"

using namespace icarus;
typedef __nv_bfloat16 bf16;

namespace {

struct Geo {
    int n1, n2, n3, q1, q2, q3;   // interior and padded (n + 2) extents
    long long N, NP;
};

Geo make_geo(int n1, int n2, int n3)
{
    Geo g;
    g.n1 = n1; g.n2 = n2; g.n3 = n3;
    g.q1 = n1 + 2; g.q2 = n2 + 2; g.q3 = n3 + 2;
    g.N = (long long)n1 * n2 * n3;
    g.NP = (long long)g.q1 * g.q2 * g.q3;
    return g;
}

__host__ __device__ __forceinline__ long long pidx(const Geo &g, int i, int j, int k)
{
    return ((long long)(k + 1) * g.q2 + (j + 1)) * g.q1 + (i + 1);
}

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// ---- forward on the 5th-generation tensor cores (tcgen05, accumulators in tensor memory) ---------
// The same y = act(conv(P(x)) + b) as an implicit GEMM D[128 voxels][O] = sum over the 27 taps and
// the input channels, one tcgen05.mma (M = 128, N = O, K = 16, BF16 in, FP32 accumulate) per tap
// and 16 channels, issued by one thread, accumulated in tensor memory.
// A tile is 128 consecutive voxels along r at fixed (j, k). Shared memory holds r-lines of the
// padded input with one halo voxel on each side (130 rows) in the no-swizzle K-major operand
// layout: a row is 16 bytes (8 channels), rows of one channel group are consecutive
// ([line][group][row][8 channels], each (line, group) block padded to 136 rows so that it starts
// on a 128-byte boundary), so 8-row core matrices are 128 bytes apart (stride offset) and channel
// groups one block apart (leading offset). The operand of tap (d1, d2, d3) is line (d2, d3)
// started d1 + 1 rows in: a 16-byte shift of the descriptor's start address, no re-staging per
// tap. A block walks the tiles of one column (i0, j) along k: the three lines (j - 1, j, j + 1) of
// a padded k index form a plane, a ring of planes holds the three a tile reads and the next ones,
// so each tile brings in one new plane (three lines instead of nine). The tensor memory
// accelerator fills each block with one 130 x 8 box of a 5-D tensor map (channel in group, group,
// i, j, k), zero beyond the padded line; the weights of all taps are staged once per block in the
// same layout ([tap][group][o][8]). Persistent blocks of 128 threads (one per SM, 208 KB of shared
// memory at C = O = 32) with two accumulators: thread 0 waits for tile k's newest plane and issues
// its MMAs into one accumulator; once tile k-1's MMAs are done it starts the copy of a plane
// several tiles ahead into the slot tile k-1 freed, and every thread reads its row of tile k-1's D
// (tcgen05.ld), adds the bias, applies the ReLU and stores, while the tensor core works on tile k.
// All waits are bounded: on expiry the block records the failure in tc_status and stops.
__device__ int tc_status;
__device__ float tc_zero_bias[32];
bool tc_host_error = false;

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr(dst)), "l"(src), "r"(bytes) : "memory");
}

// shared-memory matrix descriptor: no swizzle, start / leading / stride byte offsets in 16-byte units
__device__ __forceinline__ uint64_t umma_desc(uint32_t start, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((start & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, N = O, M = 128
template <int O> __device__ __forceinline__ uint32_t umma_idesc()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(O >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit = 1 << 22)
{
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// self-test of the bounded wait: one barrier expecting one arrival, given it (arrive = 1) or not
// (arrive = 0: nothing ever completes the phase); an expired wait records the failure in tc_status
__global__ void k_wait_selftest(int arrive, int limit)
{
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = saddr(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(b) : "memory");
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(b, 0, limit)) atomicExch(&tc_status, 1);
}

// one (line, channel group) block: 130 rows of 16 bytes, padded to 136 rows so that every block
// (a tensor-copy destination) starts on a 128-byte boundary; a k-plane is the three lines
// (j - 1, j, j + 1) of one padded k index; a ring of TC_RING planes holds a tile's three and the
// next ones in flight
constexpr int TC_BLOCK = 136 * 16;
constexpr int TC_KC = 8;                                     // tiles (k steps) per work item
constexpr int TC_RING = 6;                                   // k-planes in shared memory
template <int C> __host__ __device__ constexpr int tc_plane_bytes() { return 3 * (C / 8) * TC_BLOCK; }
template <int C, int O> __host__ __device__ constexpr int tc_b_bytes() { return 27 * (C / 8) * O * 16; }
// (+ 128 B to align the start to 128 bytes, 128 B of barriers, + 1 KB of slack after the weights)
template <int C, int O> __host__ __device__ constexpr int tc_smem_bytes()
{
    return 128 + 128 + TC_RING * tc_plane_bytes<C>() + tc_b_bytes<C, O>() + 1024;
}

// padded k-plane kp of column (i0, j) into dst by the tensor memory accelerator: per line and
// channel group one box of 130 rows x 8 channels (tensor map dims: channel in group, group, i, j, k
// of the padded grid); rows past the padded line are zero-filled; completion counted on bar
template <int C>
__device__ __forceinline__ void tc_load_plane(const CUtensorMap *tm, int i0, int j, int kp, int coff, unsigned char *dst,
                                              uint32_t bar)
{
    constexpr int G = C / 8;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(3 * G * 130 * 16)
                 : "memory");
#pragma unroll
    for (int jj = 0; jj < 3; ++jj)
#pragma unroll
        for (int grp = 0; grp < G; ++grp)
            asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n"
                         ::"r"(saddr(dst + (jj * G + grp) * TC_BLOCK)), "l"(tm), "r"(0), "r"(grp), "r"(i0 + coff),
                         "r"(j + jj + coff), "r"(kp + coff), "r"(bar)
                         : "memory");
}

template <int O> __device__ __forceinline__ void tc_ld(uint32_t ta, uint32_t *r)
{
    if constexpr (O == 32) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                     "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                       "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                       "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                       "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                     : "r"(ta));
    } else {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                       "=r"(r[14]), "=r"(r[15])
                     : "r"(ta));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// row 32 warp + lane of tile (i0, j, k): D from tensor memory, bias, ReLU, stores
template <int C, int O, int ACT>
__device__ __forceinline__ void tc_epilogue(const Geo &g, uint32_t ta, int i0, int j, int k, const float *__restrict__ b,
                                            bf16 *out_pad, float *out_f)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t r[O];
    tc_ld<O>(ta, r);
    const int i = i0 + 32 * warp + lane;
    if (i >= g.n1) return;
    float v[O];
#pragma unroll
    for (int e = 0; e < O; ++e) {
        v[e] = __uint_as_float(r[e]) + b[e];
        if (ACT) v[e] = fmaxf(v[e], 0.f);
    }
    if (out_pad) {
        uint32_t pk[O / 2];
#pragma unroll
        for (int e = 0; e < O / 2; ++e) pk[e] = pack2(__float2bfloat16_rn(v[2 * e]), __float2bfloat16_rn(v[2 * e + 1]));
        uint4 *dst = reinterpret_cast<uint4 *>(out_pad + pidx(g, i, j, k) * O);
#pragma unroll
        for (int e = 0; e < O / 8; ++e) dst[e] = make_uint4(pk[4 * e], pk[4 * e + 1], pk[4 * e + 2], pk[4 * e + 3]);
    }
    if (out_f) {
        float4 *dst = reinterpret_cast<float4 *>(out_f + (((long long)k * g.n2 + j) * g.n1 + i) * O);
#pragma unroll
        for (int e = 0; e < O / 4; ++e) dst[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
    }
}

template <int C, int O, int ACT>
__global__ void __launch_bounds__(128, 1) k_conv_fwd_tc(const __grid_constant__ CUtensorMap tm_in, Geo g,
                                                        const bf16 *__restrict__ w, const float *__restrict__ b,
                                                        bf16 *out_pad, float *out_f, int coff)
{
    constexpr int G = C / 8, PB = tc_plane_bytes<C>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // from the first 128-byte boundary: [MMA barriers 0, 1 | plane barriers | tensor-memory
    // address | flag | to 128 B][k-plane ring][weights]
    unsigned char *smem = smem_raw + ((128u - (saddr(smem_raw) & 127u)) & 127u);
    unsigned char *sA = smem + 128;
    unsigned char *sB = sA + TC_RING * PB;
    const uint32_t mbar0 = saddr(smem), full0 = saddr(smem + 16);   // barrier q at + 8 q
    const uint32_t slot = saddr(smem + 16 + 8 * TC_RING);
    volatile int *flag = reinterpret_cast<volatile int *>(smem + 20 + 8 * TC_RING);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tpl = (g.n1 + 127) / 128, ncol = tpl * g.n2, nchunk = (g.n3 + TC_KC - 1) / TC_KC;
    const int nitems = ncol * nchunk;

    for (int q = tid; q < 27 * G * O; q += blockDim.x) {     // weights: q = (t * G + grp) * O + o
        const int o = q % O, tg = q / O, grp = tg % G, t = tg / G;
        cp_async16(sB + q * 16, w + ((long long)o * 27 + t) * C + grp * 8, 16);
    }
    if (warp == 0) {                                          // two accumulators of O columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "n"(2 * O) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < 2; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar0 + 8 * q) : "memory");
        for (int q = 0; q < TC_RING; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(full0 + 8 * q) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(&tm_in) : "memory");
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(smem + 16 + 8 * TC_RING);
    const uint32_t idesc = umma_idesc<O>();
    const uint64_t dA = umma_desc(saddr(sA), TC_BLOCK, 128), dB = umma_desc(saddr(sB), O * 16, 128);
    uint32_t fpar = 0, mpar = 0;                        // barrier phases to wait for, one bit each
    int acc = 0;                                        // accumulator of the next tile
    bool failed = false;
    // a work item: column (i0, j), tiles k0 .. k1 - 1 walked in k; tile k reads padded planes
    // k, k + 1, k + 2 (ring slot: plane index mod TC_RING); after tile k-1's MMAs, plane
    // k + TC_RING - 1 goes into the slot plane k - 1 held, TC_RING - 3 tiles ahead of its first
    // use. Tile k's MMAs overlap tile k-1's stores.
    for (int item = blockIdx.x; item < nitems && !failed; item += gridDim.x) {
        const int col = item % ncol, chunk = item / ncol;
        const int i0 = (col % tpl) * 128, j = col / tpl, k0 = chunk * TC_KC;
        const int k1 = min(k0 + TC_KC, g.n3);
        if (tid == 0)
            for (int kp = k0; kp < k0 + TC_RING - 1 && kp <= k1 + 1; ++kp)
                tc_load_plane<C>(&tm_in, i0, j, kp, coff, sA + (kp % TC_RING) * PB, full0 + 8 * (kp % TC_RING));
        for (int k = k0; k <= k1; ++k) {                  // k = k1: drain (stores of tile k1 - 1)
            if (tid == 0) {
                int ok = 1;
                if (k < k1) {
                    for (int kp = (k == k0 ? k : k + 2); kp <= k + 2 && ok; ++kp) {
                        const int sl = kp % TC_RING;
                        ok = mbar_wait(full0 + 8 * sl, (fpar >> sl) & 1) ? 1 : 0;
                        fpar ^= 1u << sl;
                    }
                    if (ok) {
                        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                        uint64_t pl[3];                       // 16-byte units of planes k, k+1, k+2
#pragma unroll
                        for (int q = 0; q < 3; ++q) pl[q] = (uint64_t)(((k + q) % TC_RING) * (PB / 16));
                        const uint32_t td = tmem + (uint32_t)(O * acc);
#pragma unroll
                        for (int t = 0; t < 27; ++t) {
                            const int d1 = t % 3, d2 = (t / 3) % 3, d3 = t / 9;   // shifts + 1
#pragma unroll
                            for (int ks = 0; ks < C / 16; ++ks) {
                                const uint64_t ad = dA + pl[d3] + (uint64_t)((d2 * G + 2 * ks) * (TC_BLOCK / 16) + d1);
                                const uint64_t bd = dB + (uint64_t)((t * G + 2 * ks) * O);
                                const uint32_t en = (t | ks) ? 1u : 0u;
                                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(td),
                                             "l"(ad), "l"(bd), "r"(idesc), "r"(en)
                                             : "memory");
                            }
                        }
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                                     ::"r"(mbar0 + 8 * acc) : "memory");
                    }
                }
                if (ok && k > k0) {                       // tile k-1's MMAs
                    ok = mbar_wait(mbar0 + 8 * (acc ^ 1), (mpar >> (acc ^ 1)) & 1) ? 1 : 0;
                    mpar ^= 1u << (acc ^ 1);
                }
                // plane k + TC_RING - 1 into plane k - 1's slot (free: its last reader, tile k-1, is
                // done; at k0 that slot was not filled by the opening loads)
                const int kn = k + TC_RING - 1;
                if (ok && kn <= k1 + 1)
                    tc_load_plane<C>(&tm_in, i0, j, kn, coff, sA + (kn % TC_RING) * PB, full0 + 8 * (kn % TC_RING));
                *flag = ok;
            }
            __syncthreads();
            if (*flag == 0) {                             // a wait expired: give up
                if (tid == 0) atomicExch(&tc_status, 1);
                failed = true;
                break;
            }
            if (k > k0) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                tc_epilogue<C, O, ACT>(g, tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(O * (acc ^ 1)), i0, j, k - 1,
                                       b, out_pad, out_f);
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();                              // accumulator acc ^ 1 is free again
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (k < k1) acc ^= 1;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(2 * O) : "memory");
}

// ---- padding and its adjoint ------------------------------------------------------------------
template <typename T>
__global__ void k_pad_fill(Geo g, T *buf, int C)
{
    const unsigned int q = blockIdx.x * blockDim.x + threadIdx.x;     // padded cells < 2^31
    if (q >= (unsigned int)g.NP) return;
    const unsigned int r = q / (unsigned int)g.q1;
    const int i = (int)(q % (unsigned int)g.q1) - 1, j = (int)(r % (unsigned int)g.q2) - 1,
              k = (int)(r / (unsigned int)g.q2) - 1;
    if (i >= 0 && i < g.n1 && j >= 0 && j < g.n2 && k >= 0 && k < g.n3) return;
    const int si = min(max(i, 0), g.n1 - 1), sj = min(max(j, 0), g.n2 - 1), sk = (k + g.n3) % g.n3;
    const long long src = pidx(g, si, sj, sk);
    if ((C * sizeof(T)) % 16 == 0) {                  // whole cells in 16-byte pieces
        const uint4 *s = reinterpret_cast<const uint4 *>(buf + src * C);
        uint4 *d = reinterpret_cast<uint4 *>(buf + (long long)q * C);
        for (int c = 0; c < (int)(C * sizeof(T) / 16); ++c) d[c] = s[c];
    } else {
        for (int c = 0; c < C; ++c) buf[(long long)q * C + c] = buf[src * C + c];
    }
}

// add every ghost cell's gradient to the interior cell it copies (in place, interior = result)
__global__ void k_pad_fold(Geo g, float *buf, int C)
{
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= g.NP) return;
    int ip = (int)(q % g.q1);
    long long r = q / g.q1;
    int jp = (int)(r % g.q2), kp = (int)(r / g.q2);
    int i = ip - 1, j = jp - 1, k = kp - 1;
    if (i >= 0 && i < g.n1 && j >= 0 && j < g.n2 && k >= 0 && k < g.n3) return;
    int si = min(max(i, 0), g.n1 - 1), sj = min(max(j, 0), g.n2 - 1), sk = (k + g.n3) % g.n3;
    long long src = pidx(g, si, sj, sk);
    for (int c = 0; c < C; ++c) atomicAdd(&buf[src * C + c], buf[q * C + c]);
}

// ---- gradient w.r.t. the pre-activation, bias gradient ------------------------------------------
// dout: fp32, padded layout [NP][O] (pad = 1) or interior [N][O] (pad = 0); act_out: the layer's
// activated output (bf16 padded) for the ReLU mask (null for a linear layer). dpre: bf16 padded
// with zero ghosts. db += sum over voxels.
template <int O>
__global__ void __launch_bounds__(256) k_dpre(Geo g, const float *__restrict__ dout, int dout_padded,
                                              const bf16 *__restrict__ act_out, bf16 *dpre, float *db)
{
    __shared__ float sdb[O];
    if (threadIdx.x < O) sdb[threadIdx.x] = 0.f;
    __syncthreads();
    const unsigned int q = blockIdx.x * blockDim.x + threadIdx.x;   // padded cells < 2^31
    const bool live = q < (unsigned int)g.NP;
    float d[O];
#pragma unroll
    for (int o = 0; o < O; ++o) d[o] = 0.f;
    if (live) {
        const unsigned int r = q / (unsigned int)g.q1;
        const int i = (int)(q - r * (unsigned int)g.q1) - 1, j = (int)(r % (unsigned int)g.q2) - 1,
                  k = (int)(r / (unsigned int)g.q2) - 1;
        if (i >= 0 && i < g.n1 && j >= 0 && j < g.n2 && k >= 0 && k < g.n3) {
            const long long s = dout_padded ? (long long)q : ((long long)k * g.n2 + j) * g.n1 + i;
            const float4 *src = reinterpret_cast<const float4 *>(dout + s * O);
#pragma unroll
            for (int e = 0; e < O / 4; ++e) {
                const float4 v = src[e];
                d[4 * e] = v.x; d[4 * e + 1] = v.y; d[4 * e + 2] = v.z; d[4 * e + 3] = v.w;
            }
            if (act_out) {
                const uint4 *am = reinterpret_cast<const uint4 *>(act_out + (long long)q * O);
#pragma unroll
                for (int e = 0; e < O / 8; ++e) {
                    const uint4 a = am[e];
                    const uint32_t wds[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                    for (int h = 0; h < 8; ++h) {
                        const float av = __uint_as_float((wds[h >> 1] >> (16 * (h & 1))) << 16);
                        if (!(av > 0.f)) d[8 * e + h] = 0.f;
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < O; ++o) d[o] = __bfloat162float(__float2bfloat16_rn(d[o]));
        }
        uint32_t pk[O / 2];
#pragma unroll
        for (int e = 0; e < O / 2; ++e) pk[e] = pack2(__float2bfloat16_rn(d[2 * e]), __float2bfloat16_rn(d[2 * e + 1]));
        uint4 *dst = reinterpret_cast<uint4 *>(dpre + (long long)q * O);
#pragma unroll
        for (int e = 0; e < O / 8; ++e) dst[e] = make_uint4(pk[4 * e], pk[4 * e + 1], pk[4 * e + 2], pk[4 * e + 3]);
    }
    // db: warp sums per channel, one shared atomic per warp and channel
#pragma unroll
    for (int o = 0; o < O; ++o) {
        float v = d[o];
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) v += __shfl_xor_sync(0xffffffffu, v, sh);
        if ((threadIdx.x & 31) == 0) atomicAdd(&sdb[o], v);
    }
    __syncthreads();
    if (threadIdx.x < O) atomicAdd(&db[threadIdx.x], sdb[threadIdx.x]);
}

// ---- weight gradient on the 5th-generation tensor cores ------------------------------------------
// dw[o][t][c] += sum over interior voxels x of dpre[x][o] in[x + off_t][c], tap t = (d1, d2, d3).
// With the output gradients zero on the ghost cells, one contiguous range of padded positions p
// serves every tap: writing x = p - d1, the sum is sum_p dpre[p - d1][o] in[p + off(d2, d3)][c],
// off(d2, d3) = (d3 q2 + d2) q1 (the line of the tap), over p in [(q2 + 1) q1, last interior + 2).
// As one GEMM: D[(d1, o)][(line, c)] = sum_p A[(d1, o)][p] B[(line, c)][p], M = 3 O rows (padded
// to 128), N = 9 C columns (the nine lines (d2, d3); two MMAs of N = 144 at C = 32), K = the
// positions, split into one contiguous range per block (one block per SM; whole 64-position
// stages, so only the last block runs past the range, where dpre is zero: every padded position
// after the last interior cell is a ghost). The accumulator lives in tensor memory over the
// block's whole range and is written out once as a partial sum; a second kernel adds the blocks'
// partials into dw.
// A stage's raw rows (66 rows of dpre, 64 rows of each of the nine input lines, channels-last)
// arrive by ten tensor-memory-accelerator box copies with the 64-byte (32-byte at 16 channels)
// swizzle, three stages ahead in a ring of four buffers. Each stage is transposed into the K-major
// operand layout of the forward kernels (a 16-byte row holds 8 consecutive positions of one
// channel) by ldmatrix.trans, warp w taking the 8 x 8 tiles of positions 8 w .. 8 w + 7 (one tile
// per channel group and matrix of the ldmatrix; the swizzle puts the eight rows of a tile in
// distinct banks), once the previous stage's MMAs, which read the single operand buffer, have
// committed. Bounded waits; on expiry the block records the failure in tc_status.
constexpr int WG_KS = 64;                                          // positions per stage
constexpr int WG_RING = 4;                                         // raw-row buffers (fetch distance 3)
template <int C> __host__ __device__ constexpr int wg_a_bytes() { return (WG_KS / 8) * 128 * 16; }
template <int C> __host__ __device__ constexpr int wg_b_bytes() { return (WG_KS / 8) * 9 * C * 16; }
// raw rows of dpre (rounded up to the 1024-byte alignment of a swizzled copy) and of the lines
template <int O> __host__ __device__ constexpr int wg_ra_bytes() { return ((WG_KS + 2) * 2 * O + 1023) / 1024 * 1024; }
template <int C> __host__ __device__ constexpr int wg_rb_bytes() { return 9 * WG_KS * 2 * C; }
// [raw rows x WG_RING][operands][barriers: 128] + 1024 B of alignment
template <int C, int O> __host__ __device__ constexpr int wg_smem_bytes()
{
    return 1024 + WG_RING * (wg_ra_bytes<O>() + wg_rb_bytes<C>()) + wg_a_bytes<C>() + wg_b_bytes<C>() + 128;
}

// byte offset of 16-byte piece grp of raw row r (G pieces of 16 bytes per row) in a 1024-byte
// aligned buffer written by a swizzled tensor copy: the piece index is XORed with address bits 7-8
// (64-byte swizzle, G = 4) or bit 7 (32-byte swizzle, G = 2)
template <int G> __device__ __forceinline__ int wg_piece(int r, int grp)
{
    return r * (16 * G) + 16 * (grp ^ (G == 4 ? (r >> 1) & 3 : (r >> 2) & 1));
}

// the raw rows of the stage starting at p0: dpre rows p0 - 1 .. p0 + 64 into ra, rows p0 + off(line)
// .. + 63 of the input into rb (line after line); rows past the arrays read as zero
template <int C, int O>
__device__ __forceinline__ void wg_fetch(const CUtensorMap *ta, const CUtensorMap *tb, const Geo &g, long long p0,
                                         unsigned char *ra, unsigned char *rb, uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
                 "r"((WG_KS + 2) * 2 * O + 9 * WG_KS * 2 * C)
                 : "memory");
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
                 ::"r"(saddr(ra)), "l"(ta), "r"(0), "r"((int)(p0 - 1)), "r"(bar)
                 : "memory");
#pragma unroll
    for (int line = 0; line < 9; ++line) {
        const long long row = p0 + ((long long)(line / 3 - 1) * g.q2 + (line % 3 - 1)) * g.q1;
        asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
                     ::"r"(saddr(rb + line * WG_KS * 2 * C)), "l"(tb), "r"(0), "r"((int)row), "r"(bar)
                     : "memory");
    }
}

// the 8 x 8 tiles of position group kc (this warp's) of one operand, sel = 0 .. NSEL - 1, channel
// groups 0 .. G - 1: raw rows row0(sel) + 8 kc .. + 7, transposed by ldmatrix.trans (matrix =
// channel group) into the core matrices at dst + kc kstride + (sel G + grp) 128
template <int G, int NSEL, typename Row0>
__device__ __forceinline__ void wg_transpose(const unsigned char *raw, Row0 row0, unsigned char *dst, int kstride, int kc,
                                             int lane)
{
    const int m = (lane >> 3) % G, r = lane & 7;
    const uint32_t base = saddr(raw);
    uint32_t *out = reinterpret_cast<uint32_t *>(dst + kc * kstride) + lane;
#pragma unroll
    for (int sel = 0; sel < NSEL; ++sel) {
        const uint32_t a = base + (uint32_t)wg_piece<G>(row0(sel) + 8 * kc + r, m);
        if constexpr (G == 4) {
            uint32_t t[4];
            asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                         : "=r"(t[0]), "=r"(t[1]), "=r"(t[2]), "=r"(t[3]) : "r"(a));
#pragma unroll
            for (int j = 0; j < 4; ++j) out[(sel * G + j) * 32] = t[j];
        } else {
            uint32_t t[2];
            asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(t[0]), "=r"(t[1]) : "r"(a));
#pragma unroll
            for (int j = 0; j < 2; ++j) out[(sel * G + j) * 32] = t[j];
        }
    }
}

template <int C, int O>
__global__ void __launch_bounds__(256, 1) k_conv_wgrad_tc(const __grid_constant__ CUtensorMap tm_a,
                                                          const __grid_constant__ CUtensorMap tm_b, Geo g,
                                                          float *__restrict__ part, long long p_lo, long long p_hi,
                                                          long long chunk)
{
    constexpr int NC = 9 * C, NH = NC > 256 ? 2 : 1, NN = NC / NH, TCOLS = NC > 256 ? 512 : 256;
    constexpr int AB = wg_a_bytes<C>(), KC = WG_KS / 8;
    constexpr int RAB = wg_ra_bytes<O>(), RSB = RAB + wg_rb_bytes<C>();
    static_assert(NN % 16 == 0 && NN <= 256 && 3 * O <= 128, "tile shape");
    static_assert(KC == 8 && (O == 16 || O == 32) && (C == 16 || C == 32), "one warp per position group of 8");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *raw0 = smem_raw + ((1024u - (saddr(smem_raw) & 1023u)) & 1023u);
    // [raw rows x WG_RING][operands A | B][MMA barrier | ring barriers | tensor-memory address | flag]
    unsigned char *sA = raw0 + WG_RING * RSB, *sB = sA + AB, *hdr = sB + wg_b_bytes<C>();
    const uint32_t mbar = saddr(hdr), full0 = saddr(hdr + 8), slot = saddr(hdr + 8 + 8 * WG_RING);
    volatile int *flag = reinterpret_cast<volatile int *>(hdr + 12 + 8 * WG_RING);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long b0 = p_lo + (long long)blockIdx.x * chunk, b1 = min(b0 + chunk, p_hi);
    const int nst = b1 > b0 ? (int)((b1 - b0 + WG_KS - 1) / WG_KS) : 0;
    // rows 3 O .. 127 of A (no output) are zero
    for (int q = tid; q < KC * (128 - 3 * O) * 4; q += blockDim.x) {
        const int w4 = q % 4, rq = q / 4, row = 3 * O + rq % (128 - 3 * O), kc = rq / (128 - 3 * O);
        reinterpret_cast<uint32_t *>(sA + kc * 2048 + row * 16)[w4] = 0u;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "n"(TCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    int issued = 0;                                                // stages whose copies were started
    if (tid == 0) {
        for (int q = 0; q <= WG_RING; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar + 8 * q) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(&tm_a) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(&tm_b) : "memory");
        for (; issued < WG_RING - 1 && issued < nst; ++issued)
            wg_fetch<C, O>(&tm_a, &tm_b, g, b0 + (long long)issued * WG_KS, raw0 + issued * RSB, raw0 + issued * RSB + RAB,
                           full0 + 8 * issued);
        *flag = 1;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(hdr + 8 + 8 * WG_RING);
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    bool failed = false;
    int consumed = 0;                                              // stages whose copies were waited for
    for (int s = 0; s < nst; ++s) {
        const int q = s % WG_RING;
        unsigned char *ra = raw0 + q * RSB, *rb = ra + RAB;
        const bool got = mbar_wait(full0 + 8 * q, (uint32_t)((s / WG_RING) & 1));   // every thread: its view of the copy
        if (s >= 1 && tid == 0)                                    // stage s - 1's MMAs read the operands
            *flag = mbar_wait(mbar, (uint32_t)((s - 1) & 1)) ? 1 : 0;
        if (__syncthreads_or(!got) || *flag == 0) { failed = true; break; }
        consumed = s + 1;
        if (tid == 0 && issued < nst) {                            // into the buffer stage s - 1 left
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            const int qn = issued % WG_RING;
            wg_fetch<C, O>(&tm_a, &tm_b, g, b0 + (long long)issued * WG_KS, raw0 + qn * RSB, raw0 + qn * RSB + RAB,
                           full0 + 8 * qn);
            ++issued;
        }
        wg_transpose<O / 8, 3>(ra, [](int sel) { return 2 - sel; }, sA, 2048, warp, lane);
        wg_transpose<C / 8, 9>(rb, [](int line) { return line * WG_KS; }, sB, NC * 16, warp, lane);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();                                           // operands written, raw rows read
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < KC / 2; ++ks) {
#pragma unroll
                for (int h = 0; h < NH; ++h) {
                    const uint64_t ad = umma_desc(saddr(sA) + ks * 2 * 2048, 2048, 128);
                    const uint64_t bd = umma_desc(saddr(sB) + ks * 2 * (NC * 16) + h * (NN / 8) * 128, NC * 16, 128);
                    const uint32_t en = (s | ks) ? 1u : 0u;
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + (uint32_t)(h * NN)),
                                 "l"(ad), "l"(bd), "r"(idesc), "r"(en)
                                 : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar) : "memory");
        }
    }
    if (tid == 0) {
        // copies started but not waited for (a failed block) end before the block does
        for (int t = failed ? consumed : issued; t < issued; ++t) mbar_wait(full0 + 8 * (t % WG_RING), (uint32_t)((t / WG_RING) & 1));
        if (!failed && nst > 0) *flag = mbar_wait(mbar, (uint32_t)((nst - 1) & 1)) ? 1 : 0;
    }
    __syncthreads();
    if (*flag == 0) failed = true;
    if (failed) {
        if (tid == 0) atomicExch(&tc_status, 1);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int qd = warp & 3, hf = warp >> 2, row = 32 * qd + lane;
        float *dst = part + ((long long)blockIdx.x * 3 * O + row) * NC;
        for (int c0 = hf * (NC / 2); c0 < (hf + 1) * (NC / 2); c0 += 8) {
            uint32_t r[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                         : "r"(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (row < 3 * O) {
#pragma unroll
                for (int e = 0; e < 8; ++e) dst[c0 + e] = nst > 0 ? __uint_as_float(r[e]) : 0.f;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(TCOLS) : "memory");
}

// dw[o][t][c] += the blocks' partial sums of row (d1 + 1) O + o, column line C + c, t = 3 line + d1 + 1
template <int C, int O>
__global__ void k_wgrad_reduce(const float *__restrict__ part, int nblk, float *dw)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= O * 27 * C) return;
    const int c = e % C, t = (e / C) % 27, o = e / (27 * C);
    const int row = (t % 3) * O + o, col = (t / 3) * C + c;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[((long long)b * 3 * O + row) * (9 * C) + col];
    dw[e] += s;
}


// ---- normalisation, loss, correction, optimiser --------------------------------------------------
// x[z][c] = (U[c][v] - mean[c][i]) / scale[c][i] for c < 8, 0 for c in [8, 16)
__global__ void k_norm_in(Geo g, const double *__restrict__ U, const double *__restrict__ mean,
                          const double *__restrict__ scale, bf16 *x)
{
    const unsigned int v = blockIdx.x * blockDim.x + threadIdx.x;     // voxels < 2^31
    if (v >= (unsigned int)g.N) return;
    const unsigned int r = v / (unsigned int)g.n1;
    const int i = (int)(v % (unsigned int)g.n1), j = (int)(r % (unsigned int)g.n2), k = (int)(r / (unsigned int)g.n2);
    // (U - mean) in double, the division by the scale in single precision (the result is BF16)
    uint32_t pk[8];
#pragma unroll
    for (int c = 0; c < NV; c += 2) {
        const float a = (float)(U[c * g.N + v] - mean[c * g.n1 + i]) / (float)scale[c * g.n1 + i];
        const float b = (float)(U[(c + 1) * g.N + v] - mean[(c + 1) * g.n1 + i]) / (float)scale[(c + 1) * g.n1 + i];
        pk[c / 2] = pack2(__float2bfloat16_rn(a), __float2bfloat16_rn(b));
    }
#pragma unroll
    for (int c = 4; c < 8; ++c) pk[c] = 0u;            // channels 8 .. 15 are zero padding
    uint4 *d = reinterpret_cast<uint4 *>(x + pidx(g, i, j, k) * 16);
    d[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    d[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

// loss = mean over voxels and the 8 fields of (y - dU / oscale)^2; dy = its gradient
__global__ void __launch_bounds__(256) k_mse(Geo g, const float *__restrict__ y, const double *__restrict__ dU,
                                             const double *__restrict__ oscale, float *dy, double *loss)
{
    __shared__ double red[8];
    const unsigned int v = blockIdx.x * blockDim.x + threadIdx.x;   // voxels < 2^31
    double s = 0.0;
    if (v < (unsigned int)g.N) {
        const int i = (int)(v % (unsigned int)g.n1);
        // per element in single precision (the network's own precision), the sum in double
        const float norm = (float)(1.0 / (8.0 * (double)g.N));
        const float4 *yv = reinterpret_cast<const float4 *>(y + (long long)v * 16);
        float4 *dv = reinterpret_cast<float4 *>(dy + (long long)v * 16);
        float e[NV];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float4 yy = yv[h];
            const float ya[4] = {yy.x, yy.y, yy.z, yy.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 4 * h + q;
                e[c] = ya[q] - (float)dU[(long long)c * g.N + v] / (float)oscale[c * g.n1 + i];
                s += (double)(e[c] * e[c]);
            }
        }
        s *= (double)norm;
        dv[0] = make_float4(2.f * e[0] * norm, 2.f * e[1] * norm, 2.f * e[2] * norm, 2.f * e[3] * norm);
        dv[1] = make_float4(2.f * e[4] * norm, 2.f * e[5] * norm, 2.f * e[6] * norm, 2.f * e[7] * norm);
        dv[2] = make_float4(0.f, 0.f, 0.f, 0.f);
        dv[3] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        atomicAdd(loss, t);
    }
}

// correction in the solver's padded FP64 layout: U[c] += y[c] * oscale[c][i]
__global__ void k_apply(Params P, Geo g, const float *__restrict__ y, const double *__restrict__ oscale, double *U)
{
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.N) return;
    const int i = (int)(v % g.n1);
    const long long r = v / g.n1;
    const int j = (int)(r % g.n2), k = (int)(r / g.n2);
    const long long c = cidx(P, i, j, k);
    for (int f = 0; f < NV; ++f) U[f * P.nt + c] += (double)y[v * 16 + f] * oscale[f * g.n1 + i];
}

__global__ void k_unpack_dU(Geo g, const float *__restrict__ y, const double *__restrict__ oscale, double *dU)
{
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.N) return;
    const int i = (int)(v % g.n1);
    for (int f = 0; f < NV; ++f) dU[f * g.N + v] = (double)y[v * 16 + f] * oscale[f * g.n1 + i];
}

// Adam (FP32 master weights) and refresh of the BF16 copies w[O][27][C] and wt[C][27][O]
__global__ void k_adam(int n, float *w, float *m, float *v, const float *grad, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    float gq = grad[q];
    float mq = b1 * m[q] + (1.f - b1) * gq;
    float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    w[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

__global__ void k_weights_bf16(int O, int C, const float *w, bf16 *wb, bf16 *wt)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= O * 27 * C) return;
    int c = q % C, t = (q / C) % 27, o = q / (27 * C);
    bf16 x = __float2bfloat16_rn(w[q]);
    wb[q] = x;
    wt[((long long)c * 27 + (26 - t)) * O + o] = x;          // transposed, taps reversed
}

// volume-weighted 2x2x2 restriction of a fine solver state onto a coarse one (padded layouts)
__global__ void k_restrict(Params F, Params Cc, const double *__restrict__ Uf, double *Uc)
{
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (long long)Cc.n1 * Cc.n2 * Cc.n3) return;
    const int i = (int)(v % Cc.n1);
    const long long r = v / Cc.n1;
    const int j = (int)(r % Cc.n2), k = (int)(r / Cc.n2);
    double s[NV] = {0}, vs = 0.0;
    for (int q = 0; q < 8; ++q) {
        const int a = 2 * i + (q & 1), b = 2 * j + ((q >> 1) & 1), cc = 2 * k + ((q >> 2) & 1);
        const double vol = 1.0 / (F.m.iv1[a + NG] * F.m.iv2[b + NG] * F.m.iv3);
        const long long id = cidx(F, a, b, cc);
        for (int f = 0; f < NV; ++f) s[f] += vol * Uf[f * F.nt + id];
        vs += vol;
    }
    const long long id = cidx(Cc, i, j, k);
    for (int f = 0; f < NV; ++f) Uc[f * Cc.nt + id] = s[f] / vs;
}

unsigned int ccdiv(long long a, long long b) { return (unsigned int)((a + b - 1) / b); }

// layer shapes (C_in padded, C_out padded, real C_in, real C_out)
const int LC[4] = {16, 32, 32, 32}, LO[4] = {32, 32, 32, 16}, RC[4] = {8, 32, 32, 32}, RO[4] = {32, 32, 32, 8};

// tensor map of a padded channels-last BF16 activation buffer with C channels, as 5-D boxes
// (channel in group, group of 8 channels, i, j, k); encoded through the driver entry point
bool tc_tensor_map(CUtensorMap *tm, const bf16 *buf, const Geo &g, int C)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint64_t dims[5] = {8, (cuuint64_t)(C / 8), (cuuint64_t)g.q1, (cuuint64_t)g.q2, (cuuint64_t)g.q3};
    const cuuint64_t strides[4] = {16, (cuuint64_t)C * 2, (cuuint64_t)g.q1 * C * 2, (cuuint64_t)g.q1 * g.q2 * C * 2};
    const cuuint32_t box[5] = {8, 1, 130, 1, 1}, estr[5] = {1, 1, 1, 1, 1};
    return encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void *)buf, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D tensor map of a channels-last BF16 buffer [rows][ch] (ch = 16 or 32) read in boxes of
// box_rows whole rows with the 32-byte (16 channels) or 64-byte (32 channels) swizzle
bool wg_tensor_map(CUtensorMap *tm, const bf16 *buf, long long rows, int ch, int box_rows)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)ch, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ch * 2};
    const cuuint32_t box[2] = {(cuuint32_t)ch, (cuuint32_t)box_rows}, estr[2] = {1, 1};
    return encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  ch == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int C, int O, int ACT> int tc_prepare()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_conv_fwd_tc<C, O, ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem_bytes<C, O>());
    }
    return sms;
}

// persistent tcgen05 convolution over the interior of geometry g (one block per SM at most one per
// work item); the input's tensor map tm, its coordinates shifted by coff
template <int C, int O, int ACT>
void launch_conv_tc(const CUtensorMap &tm, Geo g, const bf16 *w, const float *b, bf16 *out_pad, float *out_f, int coff,
                    cudaStream_t s)
{
    const int sms = tc_prepare<C, O, ACT>();
    const long long items = (long long)((g.n1 + 127) / 128) * g.n2 * ((g.n3 + TC_KC - 1) / TC_KC);
    const unsigned int nb = (unsigned int)(items < sms ? items : sms);
    k_conv_fwd_tc<C, O, ACT><<<nb, 128, tc_smem_bytes<C, O>(), s>>>(tm, g, w, b, out_pad, out_f, coff);
}

// forward: interior voxels of g from the padded input (ghosts filled)
template <int C, int O, int ACT>
void launch_fwd_tc(Geo g, const bf16 *in, const bf16 *w, const float *b, bf16 *out_pad, float *out_f, cudaStream_t s)
{
    CUtensorMap tm;
    if (!tc_tensor_map(&tm, in, g, C)) {
        tc_host_error = true;
        return;
    }
    launch_conv_tc<C, O, ACT>(tm, g, w, b, out_pad, out_f, 0, s);
}

// data gradient as the same convolution: every padded voxel z of g (the interior of a geometry
// whose cells are g's padded cells) gets sum_t wt[c][26 - t][o] dpre[z + off_t][o], i.e.
// sum_t w[o][t][c] dpre[z - off_t][o], with zeros beyond the padded box (the tensor copies fill
// them); wt holds the transposed weights with the taps reversed
template <int CIN, int COUT>
void launch_dgrad_tc(Geo g, const bf16 *dpre, const bf16 *wt, float *din, cudaStream_t s)
{
    static float *zero_bias = nullptr;
    if (!zero_bias) cudaGetSymbolAddress((void **)&zero_bias, tc_zero_bias);
    CUtensorMap tm;
    if (!tc_tensor_map(&tm, dpre, g, CIN)) {
        tc_host_error = true;
        return;
    }
    launch_conv_tc<CIN, COUT, 0>(tm, make_geo(g.q1, g.q2, g.q3), wt, zero_bias, nullptr, din, -1, s);
}

// a tcgen05 forward block whose MMA completion wait expired, or a tensor map that could not be
// encoded (read and cleared; call after a sync)
bool tc_timed_out()
{
    if (tc_host_error) {
        tc_host_error = false;
        return true;
    }
    int v = 0;
    cudaMemcpyFromSymbol(&v, tc_status, sizeof v);
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(tc_status, &zero, sizeof zero);
    }
    return v != 0;
}

// a tensor map that could not be encoded (the affected launch was skipped): host-side, no sync
bool tc_map_failed()
{
    const bool f = tc_host_error;
    tc_host_error = false;
    return f;
}

void launch_fwd(int l, Geo g, const bf16 *in, const bf16 *w, const float *b, bf16 *out_pad, float *out_f, cudaStream_t s)
{
    if (l == 0) launch_fwd_tc<16, 32, 1>(g, in, w, b, out_pad, out_f, s);
    else if (l < 3) launch_fwd_tc<32, 32, 1>(g, in, w, b, out_pad, out_f, s);
    else launch_fwd_tc<32, 16, 0>(g, in, w, b, out_pad, out_f, s);
}

// weight gradient of geometry g: one tensor-core block per SM over its range of padded positions,
// then the reduction of the blocks' partials (part: wgrad_part_floats() floats) into dw
template <int C, int O>
void launch_wgrad_tc(Geo g, const bf16 *dpre, const bf16 *in, float *dw, float *part, cudaStream_t s)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_conv_wgrad_tc<C, O>, cudaFuncAttributeMaxDynamicSharedMemorySize, wg_smem_bytes<C, O>());
    }
    const long long p_lo = (long long)(g.q2 + 1) * g.q1;
    const long long p_hi = ((long long)g.n3 * g.q2 + g.n2) * g.q1 + g.n1 + 2;
    const long long span = p_hi - p_lo;
    const long long chunk = (span + (long long)sms * WG_KS - 1) / ((long long)sms * WG_KS) * WG_KS;
    const int nb = (int)((span + chunk - 1) / chunk);
    CUtensorMap ta, tb;
    if (!wg_tensor_map(&ta, dpre, g.NP, O, WG_KS + 2) || !wg_tensor_map(&tb, in, g.NP, C, WG_KS)) {
        tc_host_error = true;
        return;
    }
    k_conv_wgrad_tc<C, O><<<nb, 256, wg_smem_bytes<C, O>(), s>>>(ta, tb, g, part, p_lo, p_hi, chunk);
    k_wgrad_reduce<C, O><<<ccdiv(O * 27 * C, 256), 256, 0, s>>>(part, nb, dw);
}

// floats of the partial-sum buffer of launch_wgrad (one block per SM, 3 x 32 rows x 9 x 32 columns)
size_t wgrad_part_floats()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (size_t)(sms > 0 ? sms : 1) * 3 * 32 * 9 * 32;
}

void launch_wgrad(int l, Geo g, const bf16 *dpre, const bf16 *in, float *dw, float *part, cudaStream_t s)
{
    if (l == 0) launch_wgrad_tc<16, 32>(g, dpre, in, dw, part, s);
    else if (l < 3) launch_wgrad_tc<32, 32>(g, dpre, in, dw, part, s);
    else launch_wgrad_tc<32, 16>(g, dpre, in, dw, part, s);
}

void launch_dgrad(int l, Geo g, const bf16 *dpre, const bf16 *wt, float *din, cudaStream_t s)
{
    if (l == 3) launch_dgrad_tc<16, 32>(g, dpre, wt, din, s);
    else launch_dgrad_tc<32, 32>(g, dpre, wt, din, s);   // layers 1, 2 (layer 0 needs none)
}

void launch_dpre(int O, Geo g, const float *dout, int padded, const bf16 *act, bf16 *dpre, float *db, cudaStream_t s)
{
    const unsigned int nb = ccdiv(g.NP, 256);
    if (O == 32) k_dpre<32><<<nb, 256, 0, s>>>(g, dout, padded, act, dpre, db);
    else k_dpre<16><<<nb, 256, 0, s>>>(g, dout, padded, act, dpre, db);
}

}  // namespace

// ---------------------------------------------------------------------------------------------------
struct icarus_closure {
    Geo g;
    cudaStream_t stream = nullptr;
    std::vector<void *> allocs;
    float *w[4], *b[4], *mw[4], *vw[4], *mb[4], *vb[4], *dw[4], *db[4];
    bf16 *wb[4], *wt[4];
    bf16 *act[4];          // padded activations: act[0] = normalised input (16 ch), act[l] = output of layer l-1
    bf16 *dpre;            // padded, max 32 channels
    float *din;            // padded fp32, 32 channels
    float *wpart;          // partial sums of the weight-gradient blocks
    float *y, *dy;         // [N][16]
    double *mean, *scale, *oscale, *loss, *upack;
    int step = 0;
    bool have_norm = false;
};

namespace {

#define CCK(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return report_error(ICARUS_ECUDA, cudaGetErrorString(e_));            \
    } while (0)

void *cl_alloc(icarus_closure *c, size_t bytes)
{
    void *p = nullptr;
    if (cudaMalloc(&p, (bytes + 255) & ~(size_t)255) != cudaSuccess) return nullptr;
    c->allocs.push_back(p);
    return p;
}

uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double gauss(uint64_t &s)
{
    double u1 = ((splitmix(s) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    double u2 = (splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
}

int refresh_bf16(icarus_closure *c)
{
    for (int l = 0; l < 4; ++l) {
        int n = LO[l] * 27 * LC[l];
        k_weights_bf16<<<ccdiv(n, 256), 256, 0, c->stream>>>(LO[l], LC[l], c->w[l], c->wb[l], c->wt[l]);
    }
    CCK(cudaGetLastError());
    return ICARUS_OK;
}

// forward of the whole network from act[0] (already normalised and padded); y = fp32 [N][16]
void forward(icarus_closure *c)
{
    cudaStream_t s = c->stream;
    Geo g = c->g;
    for (int l = 0; l < 4; ++l) {
        if (l < 3) {
            launch_fwd(l, g, c->act[l], c->wb[l], c->b[l], c->act[l + 1], nullptr, s);
            k_pad_fill<bf16><<<ccdiv(g.NP, 256), 256, 0, s>>>(g, c->act[l + 1], LO[l]);
        } else {
            launch_fwd(l, g, c->act[l], c->wb[l], c->b[l], nullptr, c->y, s);
        }
    }
}

}  // namespace

extern "C" {

int icarus_closure_wait_selftest(int arrive, int limit)
{
    if ((arrive != 0 && arrive != 1) || limit < 1) return report_error(ICARUS_EINVAL, "arrive 0 or 1, limit >= 1");
    k_wait_selftest<<<1, 32>>>(arrive, limit);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return report_error(ICARUS_ECUDA, cudaGetErrorString(e));
    if (tc_timed_out()) return report_error(ICARUS_ETIMEOUT, "the barrier wait expired (nothing arrived)");
    return ICARUS_OK;
}

int icarus_closure_create(int n1, int n2, int n3, unsigned long long seed, void *cuda_stream, icarus_closure **out)
{
    if (n1 < 1 || n2 < 1 || n3 < 1 || !out) return report_error(ICARUS_EINVAL, "bad argument");
    icarus_closure *c = new icarus_closure();
    c->g = make_geo(n1, n2, n3);
    c->stream = (cudaStream_t)cuda_stream;
    const Geo &g = c->g;
    bool ok = true;
    uint64_t st = seed;
    for (int l = 0; l < 4; ++l) {
        const int n = LO[l] * 27 * LC[l];
        std::vector<float> hw(n, 0.f), hb(LO[l], 0.f);
        const double sd = (l < 3 ? sqrt(2.0 / (27.0 * RC[l])) : 0.1 * sqrt(1.0 / (27.0 * RC[l])));
        for (int o = 0; o < RO[l]; ++o)
            for (int t = 0; t < 27; ++t)
                for (int ci = 0; ci < RC[l]; ++ci) hw[((size_t)o * 27 + t) * LC[l] + ci] = (float)(sd * gauss(st));
        c->w[l] = (float *)cl_alloc(c, n * 4); c->mw[l] = (float *)cl_alloc(c, n * 4);
        c->vw[l] = (float *)cl_alloc(c, n * 4); c->dw[l] = (float *)cl_alloc(c, n * 4);
        c->b[l] = (float *)cl_alloc(c, LO[l] * 4); c->mb[l] = (float *)cl_alloc(c, LO[l] * 4);
        c->vb[l] = (float *)cl_alloc(c, LO[l] * 4); c->db[l] = (float *)cl_alloc(c, LO[l] * 4);
        c->wb[l] = (bf16 *)cl_alloc(c, n * 2); c->wt[l] = (bf16 *)cl_alloc(c, n * 2);
        if (!c->w[l] || !c->mw[l] || !c->vw[l] || !c->dw[l] || !c->b[l] || !c->mb[l] || !c->vb[l] || !c->db[l] ||
            !c->wb[l] || !c->wt[l]) { ok = false; break; }
        cudaMemcpy(c->w[l], hw.data(), n * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(c->b[l], hb.data(), LO[l] * 4, cudaMemcpyHostToDevice);
        cudaMemset(c->mw[l], 0, n * 4); cudaMemset(c->vw[l], 0, n * 4);
        cudaMemset(c->mb[l], 0, LO[l] * 4); cudaMemset(c->vb[l], 0, LO[l] * 4);
    }
    for (int l = 0; ok && l < 4; ++l) {
        c->act[l] = (bf16 *)cl_alloc(c, g.NP * LC[l] * 2);
        ok = c->act[l] != nullptr;
        if (ok) cudaMemset(c->act[l], 0, g.NP * LC[l] * 2);
    }
    if (ok) {
        c->dpre = (bf16 *)cl_alloc(c, g.NP * 32 * 2);
        c->din = (float *)cl_alloc(c, g.NP * 32 * 4);
        c->y = (float *)cl_alloc(c, g.N * 16 * 4);
        c->dy = (float *)cl_alloc(c, g.N * 16 * 4);
        c->mean = (double *)cl_alloc(c, 8 * n1 * 8);
        c->scale = (double *)cl_alloc(c, 8 * n1 * 8);
        c->oscale = (double *)cl_alloc(c, 8 * n1 * 8);
        c->loss = (double *)cl_alloc(c, 8);
        c->upack = (double *)cl_alloc(c, 8 * g.N * 8);
        c->wpart = (float *)cl_alloc(c, wgrad_part_floats() * 4);
        ok = c->dpre && c->din && c->y && c->dy && c->mean && c->scale && c->oscale && c->loss && c->upack && c->wpart;
    }
    if (!ok) {
        for (void *p : c->allocs) cudaFree(p);
        delete c;
        return report_error(ICARUS_ENOMEM, "closure allocation failed");
    }
    int rc = refresh_bf16(c);
    if (rc) return rc;
    CCK(cudaStreamSynchronize(c->stream));
    *out = c;
    return ICARUS_OK;
}

int icarus_closure_destroy(icarus_closure *c)
{
    if (!c) return ICARUS_OK;
    cudaStreamSynchronize(c->stream);
    for (void *p : c->allocs) cudaFree(p);
    delete c;
    return ICARUS_OK;
}

int icarus_closure_set_norm(icarus_closure *c, const double *in_mean, const double *in_scale, const double *out_scale)
{
    if (!c || !in_mean || !in_scale || !out_scale) return report_error(ICARUS_EINVAL, "NULL argument");
    const size_t n = 8 * (size_t)c->g.n1 * sizeof(double);
    CCK(cudaMemcpyAsync(c->mean, in_mean, n, cudaMemcpyHostToDevice, c->stream));
    CCK(cudaMemcpyAsync(c->scale, in_scale, n, cudaMemcpyHostToDevice, c->stream));
    CCK(cudaMemcpyAsync(c->oscale, out_scale, n, cudaMemcpyHostToDevice, c->stream));
    CCK(cudaStreamSynchronize(c->stream));
    c->have_norm = true;
    return ICARUS_OK;
}

int icarus_closure_train_step(icarus_closure *c, const double *U_in, const double *dU_target, double lr, double *loss)
{
    if (!c || !U_in || !dU_target) return report_error(ICARUS_EINVAL, "NULL argument");
    if (!c->have_norm) return report_error(ICARUS_ESTATE, "set the normalisation first");
    cudaStream_t s = c->stream;
    const Geo g = c->g;
    k_norm_in<<<ccdiv(g.N, 256), 256, 0, s>>>(g, U_in, c->mean, c->scale, c->act[0]);
    k_pad_fill<bf16><<<ccdiv(g.NP, 256), 256, 0, s>>>(g, c->act[0], 16);
    forward(c);
    if (tc_map_failed()) return report_error(ICARUS_ECUDA, "tensor map encoding failed");
    CCK(cudaMemsetAsync(c->loss, 0, 8, s));
    k_mse<<<ccdiv(g.N, 256), 256, 0, s>>>(g, c->y, dU_target, c->oscale, c->dy, c->loss);
    for (int l = 0; l < 4; ++l) {
        CCK(cudaMemsetAsync(c->dw[l], 0, LO[l] * 27 * LC[l] * 4, s));
        CCK(cudaMemsetAsync(c->db[l], 0, LO[l] * 4, s));
    }
    // layer 3 (linear): gradient from the loss; then ReLU layers with the mask of their output
    for (int l = 3; l >= 0; --l) {
        if (l == 3) launch_dpre(LO[l], g, c->dy, 0, nullptr, c->dpre, c->db[l], s);
        else launch_dpre(LO[l], g, c->din, 1, c->act[l + 1], c->dpre, c->db[l], s);
        launch_wgrad(l, g, c->dpre, c->act[l], c->dw[l], c->wpart, s);
        if (l > 0) {
            launch_dgrad(l, g, c->dpre, c->wt[l], c->din, s);
            k_pad_fold<<<ccdiv(g.NP, 256), 256, 0, s>>>(g, c->din, LC[l]);
        }
    }
    if (tc_map_failed()) return report_error(ICARUS_ECUDA, "tensor map encoding failed");   // before Adam
    c->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)c->step), c2 = 1.f - powf(b2, (float)c->step);
    for (int l = 0; l < 4; ++l) {
        int n = LO[l] * 27 * LC[l];
        k_adam<<<ccdiv(n, 256), 256, 0, s>>>(n, c->w[l], c->mw[l], c->vw[l], c->dw[l], (float)lr, b1, b2, 1e-8f, c1, c2);
        k_adam<<<1, 64, 0, s>>>(LO[l], c->b[l], c->mb[l], c->vb[l], c->db[l], (float)lr, b1, b2, 1e-8f, c1, c2);
    }
    int rc = refresh_bf16(c);
    if (rc) return rc;
    if (loss) {
        CCK(cudaMemcpyAsync(loss, c->loss, 8, cudaMemcpyDeviceToHost, s));
        CCK(cudaStreamSynchronize(s));
        if (tc_timed_out()) return report_error(ICARUS_ETIMEOUT, "tensor-core forward: MMA completion wait expired");
    }
    CCK(cudaGetLastError());
    return ICARUS_OK;
}

// correction dU [8][n3][n2][n1] (device, code units) predicted for a coarse state U (device)
int icarus_closure_predict(icarus_closure *c, const double *U_in, double *dU_out)
{
    if (!c || !U_in || !dU_out) return report_error(ICARUS_EINVAL, "NULL argument");
    if (!c->have_norm) return report_error(ICARUS_ESTATE, "set the normalisation first");
    cudaStream_t s = c->stream;
    const Geo g = c->g;
    k_norm_in<<<ccdiv(g.N, 256), 256, 0, s>>>(g, U_in, c->mean, c->scale, c->act[0]);
    k_pad_fill<bf16><<<ccdiv(g.NP, 256), 256, 0, s>>>(g, c->act[0], 16);
    forward(c);
    if (tc_map_failed()) return report_error(ICARUS_ECUDA, "tensor map encoding failed");
    k_unpack_dU<<<ccdiv(g.N, 256), 256, 0, s>>>(g, c->y, c->oscale, dU_out);
    CCK(cudaGetLastError());
    return ICARUS_OK;
}

// apply the correction to a coarse FP64 context in place: U += net(U); primitives refreshed
int icarus_closure_apply(icarus_closure *c, icarus_ctx *ctx)
{
    if (!c || !ctx) return report_error(ICARUS_EINVAL, "NULL argument");
    if (ctx->opts.precision != ICARUS_FP64) return report_error(ICARUS_EINVAL, "closure needs an FP64 context");
    if (ctx->P.n1 != c->g.n1 || ctx->P.n2 != c->g.n2 || ctx->P.n3 != c->g.n3)
        return report_error(ICARUS_EINVAL, "context grid differs from the closure grid");
    if (!c->have_norm) return report_error(ICARUS_ESTATE, "set the normalisation first");
    cudaStream_t s = ctx->stream;
    CCK(cudaStreamSynchronize(c->stream));
    ctx->ops.pack(ctx->P, ctx->U, c->upack, s);
    const Geo g = c->g;
    k_norm_in<<<ccdiv(g.N, 256), 256, 0, s>>>(g, c->upack, c->mean, c->scale, c->act[0]);
    k_pad_fill<bf16><<<ccdiv(g.NP, 256), 256, 0, s>>>(g, c->act[0], 16);
    cudaStream_t keep = c->stream;
    c->stream = s;
    forward(c);
    if (tc_map_failed()) return report_error(ICARUS_ECUDA, "tensor map encoding failed");
    c->stream = keep;
    k_apply<<<ccdiv(g.N, 256), 256, 0, s>>>(ctx->P, g, c->y, c->oscale, (double *)ctx->U);
    ctx->ops.prims(ctx->P, ctx->U, ctx->W, s);
    ctx->ops.fill_ghosts(ctx->P, ctx->U, ctx->W, 1, s);
    ctx->ops.cfl(ctx->P, ctx->W, s);
    CCK(cudaGetLastError());
    return ICARUS_OK;
}

// weights out / in as FP32 host arrays, layer by layer: w[l] [O_l][27][C_l], b[l] [O_l] with the
// padded channel counts (16/32, 32/32, 32/32, 32/16)
int icarus_closure_weights(icarus_closure *c, int layer, float *w, float *b, int set)
{
    if (!c || layer < 0 || layer > 3 || !w || !b) return report_error(ICARUS_EINVAL, "bad argument");
    const size_t n = (size_t)LO[layer] * 27 * LC[layer];
    if (set) {
        CCK(cudaMemcpy(c->w[layer], w, n * 4, cudaMemcpyHostToDevice));
        CCK(cudaMemcpy(c->b[layer], b, LO[layer] * 4, cudaMemcpyHostToDevice));
        return refresh_bf16(c);
    }
    CCK(cudaMemcpy(w, c->w[layer], n * 4, cudaMemcpyDeviceToHost));
    CCK(cudaMemcpy(b, c->b[layer], LO[layer] * 4, cudaMemcpyDeviceToHost));
    return ICARUS_OK;
}

// restriction of a fine context's state onto a coarse context (2x in every direction)
int icarus_restrict(icarus_ctx *fine, icarus_ctx *coarse)
{
    if (!fine || !coarse) return report_error(ICARUS_EINVAL, "NULL argument");
    if (fine->P.n1 != 2 * coarse->P.n1 || fine->P.n2 != 2 * coarse->P.n2 || fine->P.n3 != 2 * coarse->P.n3)
        return report_error(ICARUS_EINVAL, "fine grid must be 2x the coarse grid");
    if (fine->opts.precision == ICARUS_FP32 || coarse->opts.precision == ICARUS_FP32)
        return report_error(ICARUS_EINVAL, "restriction needs double states");
    CCK(cudaStreamSynchronize(fine->stream));
    long long n = (long long)coarse->P.n1 * coarse->P.n2 * coarse->P.n3;
    k_restrict<<<ccdiv(n, 256), 256, 0, coarse->stream>>>(fine->P, coarse->P, (const double *)fine->U, (double *)coarse->U);
    coarse->ops.prims(coarse->P, coarse->U, coarse->W, coarse->stream);
    Scalars s;
    CCK(cudaMemcpyAsync(&s, fine->sc, sizeof s, cudaMemcpyDeviceToHost, fine->stream));
    CCK(cudaStreamSynchronize(fine->stream));
    Scalars sc;
    CCK(cudaMemcpyAsync(&sc, coarse->sc, sizeof sc, cudaMemcpyDeviceToHost, coarse->stream));
    CCK(cudaStreamSynchronize(coarse->stream));
    sc.t = s.t;
    sc.done = 0;
    CCK(cudaMemcpyAsync(coarse->sc, &sc, sizeof sc, cudaMemcpyHostToDevice, coarse->stream));
    coarse->have_state = true;
    coarse->ops.fill_ghosts(coarse->P, coarse->U, coarse->W, 1, coarse->stream);
    coarse->ops.cfl(coarse->P, coarse->W, coarse->stream);
    CCK(cudaGetLastError());
    CCK(cudaStreamSynchronize(coarse->stream));
    return ICARUS_OK;
}

// one layer on host FP32 arrays (values should be BF16-representable): forward y = act(conv +
// b) and, with g = dL/dy, the gradients dx, dw, db. Channel counts C, O in {16, 32}.
int icarus_conv3d_layer(int n1, int n2, int n3, int C, int O, int act, const float *x, const float *w, const float *b,
                        const float *g, float *y, float *dx, float *dw, float *db)
{
    if ((C != 16 && C != 32) || (O != 16 && O != 32) || (C == 16 && O == 16) || n1 < 1 || n2 < 1 || n3 < 1)
        return report_error(ICARUS_EINVAL, "supported (C, O): (16, 32), (32, 32), (32, 16)");
    if ((C == 16 && act != 1) || (O == 16 && act != 0))
        return report_error(ICARUS_EINVAL, "(16, 32) layers are ReLU, (32, 16) layers are linear");
    const Geo gg = make_geo(n1, n2, n3);
    const int l = C == 16 ? 0 : (O == 16 ? 3 : 1);
    std::vector<void *> mem;
    auto A = [&](size_t bytes) { void *p = nullptr; cudaMalloc(&p, bytes); mem.push_back(p); return p; };
    bf16 *din_ = (bf16 *)A(gg.NP * C * 2), *dout_ = (bf16 *)A(gg.NP * O * 2), *wb = (bf16 *)A(O * 27 * C * 2),
         *wt = (bf16 *)A(O * 27 * C * 2), *dpre = (bf16 *)A(gg.NP * O * 2);
    float *wf = (float *)A(O * 27 * C * 4), *bf = (float *)A(O * 4), *yf = (float *)A(gg.N * O * 4),
          *gf = (float *)A(gg.N * O * 4), *dinf = (float *)A(gg.NP * C * 4), *dwf = (float *)A(O * 27 * C * 4),
          *dbf = (float *)A(O * 4), *wpart = (float *)A(wgrad_part_floats() * 4);
    int rc = ICARUS_OK;
    for (void *p : mem) if (!p) rc = report_error(ICARUS_ENOMEM, "allocation failed");
    if (!rc) {
        std::vector<bf16> hx(gg.NP * C, __float2bfloat16_rn(0.f));
        for (int k = 0; k < n3; ++k)
            for (int j = 0; j < n2; ++j)
                for (int i = 0; i < n1; ++i)
                    for (int c = 0; c < C; ++c)
                        hx[pidx(gg, i, j, k) * C + c] = __float2bfloat16_rn(x[(((size_t)k * n2 + j) * n1 + i) * C + c]);
        cudaMemcpy(din_, hx.data(), hx.size() * 2, cudaMemcpyHostToDevice);
        cudaMemcpy(wf, w, O * 27 * C * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(bf, b, O * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(gf, g, gg.N * O * 4, cudaMemcpyHostToDevice);
        cudaMemset(dwf, 0, O * 27 * C * 4);
        cudaMemset(dbf, 0, O * 4);
        k_weights_bf16<<<ccdiv(O * 27 * C, 256), 256>>>(O, C, wf, wb, wt);
        k_pad_fill<bf16><<<ccdiv(gg.NP, 256), 256>>>(gg, din_, C);
        launch_fwd(l, gg, din_, wb, bf, act ? dout_ : nullptr, yf, 0);
        if (act) k_pad_fill<bf16><<<ccdiv(gg.NP, 256), 256>>>(gg, dout_, O);
        launch_dpre(O, gg, gf, 0, act ? dout_ : nullptr, dpre, dbf, 0);
        launch_wgrad(l, gg, dpre, din_, dwf, wpart, 0);
        if (C == 32) {
            if (O == 16) launch_dgrad_tc<16, 32>(gg, dpre, wt, dinf, 0);
            else launch_dgrad_tc<32, 32>(gg, dpre, wt, dinf, 0);
        } else {
            launch_dgrad_tc<32, 16>(gg, dpre, wt, dinf, 0);
        }
        k_pad_fold<<<ccdiv(gg.NP, 256), 256>>>(gg, dinf, C);
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = report_error(ICARUS_ECUDA, cudaGetErrorString(e));
        else if (tc_timed_out()) rc = report_error(ICARUS_ETIMEOUT, "tensor-core forward: MMA completion wait expired");
        if (!rc) {
            cudaMemcpy(y, yf, gg.N * O * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(dw, dwf, O * 27 * C * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(db, dbf, O * 4, cudaMemcpyDeviceToHost);
            std::vector<float> hd(gg.NP * C);
            cudaMemcpy(hd.data(), dinf, hd.size() * 4, cudaMemcpyDeviceToHost);
            for (int k = 0; k < n3; ++k)
                for (int j = 0; j < n2; ++j)
                    for (int i = 0; i < n1; ++i)
                        for (int c = 0; c < C; ++c)
                            dx[(((size_t)k * n2 + j) * n1 + i) * C + c] = hd[pidx(gg, i, j, k) * C + c];
        }
    }
    for (void *p : mem) cudaFree(p);
    return rc;
}

}  // extern "C"
