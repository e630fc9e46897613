// icarus_fused.cuh -- one SSP-RK2 stage in ONE kernel for the single-precision arithmetic forms
// (FP32 state and MIXED): face fluxes in r, theta and phi, div B, sources and the update, with no
// flux or div-B arrays in HBM.
//
// A block owns a 32 (r) x 8 (theta) column tile and a chunk of KC phi planes and streams along
// phi: a ring of four primitive planes (tile + two-cell halo) in shared memory, a ring of three
// div-B planes, and the r / theta face fluxes of the current plane in shared memory; the phi face
// below each cell is carried in registers from the previous plane. Per plane: load plane k+2,
// div B of plane k+1, the faces of plane k, then the update of its 256 cells (the single solver's
// update_core). Ghost cells come from the ghost-fill kernels that run before the stage.
#pragma once
#include "icarus_kernels.cuh"

namespace icarus {

constexpr int FT_R = 32, FT_T = 8, FT_THREADS = FT_R * FT_T;
constexpr int FT_HR = FT_R + 4, FT_HT = FT_T + 4;              // tile with two-cell halo
constexpr int FT_DR = FT_R + 2, FT_DT = FT_T + 2;              // div-B tile (one-cell halo)
constexpr int FT_PLANE = NV * FT_HT * FT_HR;                    // floats per primitive plane
constexpr size_t FT_SMEM = sizeof(float) * (4 * FT_PLANE + 3 * FT_DT * FT_DR + NV * FT_T * (FT_R + 1) +
                                            NV * (FT_T + 1) * FT_R);

struct FusedSmem {
    float *ring, *dring, *fr, *ft;
    __device__ __forceinline__ float &w(int k, int v, int jj, int ii)
    {
        return ring[(((k + 8) & 3) * NV + v) * FT_HT * FT_HR + jj * FT_HR + ii];
    }
    __device__ __forceinline__ float &d(int k, int jj, int ii) { return dring[(((k + 9) % 3) * FT_DT + jj) * FT_DR + ii]; }
    __device__ __forceinline__ float &r(int v, int tj, int f) { return fr[(v * FT_T + tj) * (FT_R + 1) + f]; }
    __device__ __forceinline__ float &t(int v, int tjj, int ti) { return ft[(v * (FT_T + 1) + tjj) * FT_R + ti]; }
};

// face flux from the four cells around it along one direction (cells a-1, a | b, b+1)
__device__ __forceinline__ void fused_face(const Params &P, int D, const float *wm1, const float *wa, const float *wb,
                                           const float *wp1, float *f)
{
    float wl[NV], wr[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const float da = limiter<float>(P.limiter, wa[v] - wm1[v], wb[v] - wa[v]);
        const float db = limiter<float>(P.limiter, wb[v] - wa[v], wp1[v] - wb[v]);
        wl[v] = wa[v] + 0.5f * da;
        wr[v] = wb[v] - 0.5f * db;
    }
    if (not_positive(wl[0]) || not_positive(wr[0]) || not_positive(wl[4]) || not_positive(wr[4])) {
#pragma unroll
        for (int v = 0; v < NV; ++v) { wl[v] = wa[v]; wr[v] = wb[v]; }
    }
    riemann<float>(wl, wr, D, P.flux, P.phf.gamma, P.phf.igm1, f);
}

template <int STAGE, typename TS>
__global__ void __launch_bounds__(FT_THREADS, 2)
k_fused_stage(Params P, const TS *__restrict__ Us, const float *__restrict__ Ws, TS *Uo, float *__restrict__ Wo,
              int kc, int tiles_r, int tiles_t)
{
    extern __shared__ __align__(16) float fsm[];
    FusedSmem S;
    S.ring = fsm;
    S.dring = S.ring + 4 * FT_PLANE;
    S.fr = S.dring + 3 * FT_DT * FT_DR;
    S.ft = S.fr + NV * FT_T * (FT_R + 1);
    const int tid = threadIdx.x, ti = tid % FT_R, tj = tid / FT_R;
    const int bx = blockIdx.x % tiles_r, by = (blockIdx.x / tiles_r) % tiles_t, bz = blockIdx.x / (tiles_r * tiles_t);
    const int i0 = bx * FT_R, j0 = by * FT_T, k0 = bz * kc, k1 = min(k0 + kc, P.n3);
    const long long nt = P.nt;
    const MetricsT<float> &m = P.mf;
    auto load_plane = [&](int k) {
        for (int q = tid; q < FT_PLANE; q += FT_THREADS) {
            const int v = q / (FT_HT * FT_HR), rem = q % (FT_HT * FT_HR), jj = rem / FT_HR, ii = rem % FT_HR;
            const int i = min(max(i0 - 2 + ii, -NG), P.n1 + 1), j = min(max(j0 - 2 + jj, -NG), P.n2 + 1);
            S.w(k, v, jj, ii) = Ws[v * nt + cidx(P, i, j, k)];
        }
    };
    // div B of plane kp over the tile with a one-cell halo (the face-average form of k_divb)
    auto divb_plane = [&](int kp) {
        for (int q = tid; q < FT_DT * FT_DR; q += FT_THREADS) {
            const int jj = q / FT_DR, ii = q % FT_DR;
            const int i = min(max(i0 - 1 + ii, -1), P.n1), j = min(max(j0 - 1 + jj, -1), P.n2);
            const int ip = i + NG, jp = j + NG, sx = ii + 1, sy = jj + 1;
            const float d1 = (m.a1[ip + 1] * (S.w(kp, 5, sy, sx) + S.w(kp, 5, sy, sx + 1)) -
                              m.a1[ip] * (S.w(kp, 5, sy, sx - 1) + S.w(kp, 5, sy, sx))) * m.iv1[ip];
            const float d2 = (m.a2[jp + 1] * (S.w(kp, 6, sy, sx) + S.w(kp, 6, sy + 1, sx)) -
                              m.a2[jp] * (S.w(kp, 6, sy - 1, sx) + S.w(kp, 6, sy, sx))) * (m.q1[ip] * m.iv2[jp]);
            const float d3 = (S.w(kp + 1, 7, sy, sx) - S.w(kp - 1, 7, sy, sx)) * (m.q1[ip] * m.q2[jp] * m.iv3);
            S.d(kp, jj, ii) = 0.5f * (d1 + d2 + d3);
        }
    };
    auto phi_face = [&](int k, float *f) {      // face between planes k and k+1 of this thread's column
        float a[NV], b[NV], c[NV], e[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            a[v] = S.w(k - 1, v, tj + 2, ti + 2);
            b[v] = S.w(k, v, tj + 2, ti + 2);
            c[v] = S.w(k + 1, v, tj + 2, ti + 2);
            e[v] = S.w(k + 2, v, tj + 2, ti + 2);
        }
        fused_face(P, 2, a, b, c, e, f);
    };
    const bool divb = P.divb == 1;
    for (int k = k0 - 2; k <= k0 + 1; ++k) load_plane(k);
    __syncthreads();
    if (divb) { divb_plane(k0 - 1); divb_plane(k0); }
    float fp_lo[NV], fp_hi[NV];
    phi_face(k0 - 1, fp_lo);
    __syncthreads();
    double smax = 0.0;
    for (int k = k0; k < k1; ++k) {
        load_plane(k + 2);
        __syncthreads();
        if (divb) divb_plane(k + 1);
        for (int q = tid; q < FT_T * (FT_R + 1); q += FT_THREADS) {      // r faces of plane k
            const int tjj = q / (FT_R + 1), f = q % (FT_R + 1);
            float a[NV], b[NV], c[NV], e[NV], fl[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                a[v] = S.w(k, v, tjj + 2, f); b[v] = S.w(k, v, tjj + 2, f + 1);
                c[v] = S.w(k, v, tjj + 2, f + 2); e[v] = S.w(k, v, tjj + 2, f + 3);
            }
            fused_face(P, 0, a, b, c, e, fl);
#pragma unroll
            for (int v = 0; v < NV; ++v) S.r(v, tjj, f) = fl[v];
        }
        for (int q = tid; q < (FT_T + 1) * FT_R; q += FT_THREADS) {      // theta faces of plane k
            const int tjj = q / FT_R, t2 = q % FT_R;
            float a[NV], b[NV], c[NV], e[NV], fl[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                a[v] = S.w(k, v, tjj, t2 + 2); b[v] = S.w(k, v, tjj + 1, t2 + 2);
                c[v] = S.w(k, v, tjj + 2, t2 + 2); e[v] = S.w(k, v, tjj + 3, t2 + 2);
            }
            fused_face(P, 1, a, b, c, e, fl);
#pragma unroll
            for (int v = 0; v < NV; ++v) S.t(v, tjj, t2) = fl[v];
        }
        phi_face(k, fp_hi);
        __syncthreads();
        const int i = i0 + ti, j = j0 + tj;
        if (i < P.n1 && j < P.n2) {
            const DivFactors<float> dv(m, i + NG, j + NG);
            float w[NV], L[NV], dbn[7];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                w[v] = S.w(k, v, tj + 2, ti + 2);
                L[v] = dv.div(S.r(v, tj, ti), S.r(v, tj, ti + 1), S.t(v, tj, ti), S.t(v, tj + 1, ti), fp_lo[v], fp_hi[v]);
            }
            if (divb) {
                dbn[0] = S.d(k, tj + 1, ti); dbn[1] = S.d(k, tj + 1, ti + 2);
                dbn[2] = S.d(k, tj, ti + 1); dbn[3] = S.d(k, tj + 2, ti + 1);
                dbn[4] = S.d(k - 1, tj + 1, ti + 1); dbn[5] = S.d(k + 1, tj + 1, ti + 1);
            }
            float wo[NV];
            update_core<STAGE, TS, float>(P, i, j, k, w, L, dbn, Us, Uo, Wo, wo);
            if (STAGE == 2) smax = fmax(smax, cell_speed<float>(P, wo, i + NG, j + NG));
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) fp_lo[v] = fp_hi[v];
        __syncthreads();
    }
    if (STAGE == 2) {
        smax = block_max(smax);
        finish_dt(P, smax, 1);
    }
}

template <typename TS> struct FusedLaunch {
    static int kc(const Params &P) { return P.n3 >= 64 ? 16 : 8; }
    static unsigned int blocks(const Params &P)
    {
        const int c = kc(P);
        return (unsigned int)(((P.n1 + FT_R - 1) / FT_R) * ((P.n2 + FT_T - 1) / FT_T) * ((P.n3 + c - 1) / c));
    }
    static void stage(const Params &P, int st, const void *Us, const void *Ws, void *Uo, void *Wo, cudaStream_t s)
    {
        const int tr = (P.n1 + FT_R - 1) / FT_R, tt = (P.n2 + FT_T - 1) / FT_T;
        if (st == 1)
            k_fused_stage<1, TS><<<blocks(P), FT_THREADS, FT_SMEM, s>>>(P, (const TS *)Us, (const float *)Ws, (TS *)Uo,
                                                                     (float *)Wo, kc(P), tr, tt);
        else
            k_fused_stage<2, TS><<<blocks(P), FT_THREADS, FT_SMEM, s>>>(P, (const TS *)Us, (const float *)Ws, (TS *)Uo,
                                                                     (float *)Wo, kc(P), tr, tt);
    }
    static void prepare()
    {
        cudaFuncSetAttribute(k_fused_stage<1, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FT_SMEM);
        cudaFuncSetAttribute(k_fused_stage<2, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FT_SMEM);
    }
};

}  // namespace icarus
