// Training of the learned proposal's network on the GPU (the library's
// extension of the spawn step; not in the paper).
//
//   k_learn_events  training events from N(t): features, heat-bath shares of
//                   the present outputs (exact integer column weights), weight
//   k_learn_fwdbwd  per event: forward pass, masked softmax cross-entropy,
//                   backpropagation to the logits and both hidden layers
//   k_learn_abt     weight gradients C = A B^T over events (fixed order)
//   k_learn_sum     fixed-order sums (event weights, losses) in double
//   k_learn_adam    Adam update of the packed parameters
//
// Layouts: per-event arrays are feature-major ([rows][ld], event index
// fastest) so that one thread per event reads and writes coalesced.  The
// parameters are packed as w1 [H x I], b1 [H], w2 [H x H], b2 [H], w3 [G x H],
// b3 [G].  Single precision with fused multiply-adds; every sum over events
// runs in a fixed order, so gradients are deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>
#include <stdint.h>

#include "column_eval.h"
#include "kernels.h"
#include "tc_ops.h"

namespace qmc {

namespace {

constexpr int kLearnThreads = 256;

__device__ __forceinline__ int64_t abs64(int64_t v) { return v < 0 ? -v : v; }

// Output index of a destination mask among the sorted output masks, or -1.
__device__ __forceinline__ int find_output(const uint64_t* masks, const int32_t* idx, int G, uint64_t mask)
{
    int lo = 0, hi = G;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (masks[mid] < mask) lo = mid + 1; else hi = mid;
    }
    return (lo < G && masks[lo] == mask) ? idx[lo] : -1;
}

// One thread per event: record r = floor(e K / E) of the current slot (all
// records when K <= E).  Targets of the present outputs are the heat-bath
// shares float(double(w_k) / double(W)); absent outputs get -1.
__global__ void k_learn_events(LearnArgs A)
{
    const DevState* st = A.st;
    const int64_t K = st->count[st->cur];
    const int64_t E = K < A.max_events ? K : A.max_events;
    if (blockIdx.x == 0 && threadIdx.x == 0) *A.n_events = E;
    const Rec* pop = A.pop[st->cur];
    const Prog prog = prog_at(A.prog);
    const int n = A.n, G = A.G, ns = prog.h->n_stat;
    const float tf = __double2float_rn(A.t);
    const uint32_t ymask = n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = K <= A.max_events ? e : (e * K) / A.max_events;
        const Rec par = pop[r];
        const uint32_t x = (uint32_t)(par.key >> n), y = (uint32_t)(par.key & ymask);
        for (int i = 0; i < n; ++i) {
            A.feat[(int64_t)i * A.ld + e] = (float)((x >> i) & 1u);
            A.feat[(int64_t)(n + i) * A.ld + e] = (float)((y >> i) & 1u);
        }
        A.feat[(int64_t)(2 * n) * A.ld + e] = tf;
        for (int g = 0; g < G; ++g) A.target[(int64_t)g * A.ld + e] = -1.0f;
        int64_t W = 0;
        for (int k = 0; k < ns; ++k) {
            const int64_t width = prog.stat[k].end - (k ? prog.stat[k - 1].end : 0);
            if (width <= 0 || find_output(A.masks, A.idx, G, prog.stat[k].mask) < 0) continue;
            int64_t vr, vi;
            value_at_mask(prog, prog.stat[k].mask, x, y, &vr, &vi);
            W += abs64(vr) + abs64(vi);
        }
        for (int k = 0; k < ns; ++k) {
            const int64_t width = prog.stat[k].end - (k ? prog.stat[k - 1].end : 0);
            const int g = width > 0 ? find_output(A.masks, A.idx, G, prog.stat[k].mask) : -1;
            if (g < 0) continue;
            float share = 0.0f;
            if (W > 0) {
                int64_t vr, vi;
                value_at_mask(prog, prog.stat[k].mask, x, y, &vr, &vi);
                share = __double2float_rn(__ddiv_rn((double)(abs64(vr) + abs64(vi)), (double)W));
            }
            A.target[(int64_t)g * A.ld + e] = share;
        }
        A.weight[e] = W > 0 ? __ll2float_rn(abs64(par.re) + abs64(par.im)) : 0.0f;
    }
}

// Fixed-order sum of v[0..E) in double into *out (one CTA).
__global__ void __launch_bounds__(1024) k_learn_sum(const float* __restrict__ v, const int64_t* n_events, int64_t E_fixed,
                                                    double* out)
{
    __shared__ double part[1024];
    const int64_t E = n_events ? *n_events : E_fixed;
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < E; e += 1024) s += (double)v[e];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

// One thread per event: forward pass, loss omega_e CE_e (omega_e = weight /
// sum of weights), dL/dz, dL/dh2 and dL/dh1 (ReLU derivative 0 at 0).
__global__ void __launch_bounds__(kLearnThreads) k_learn_fwdbwd(LearnGrad A)
{
    const int I = A.I, H = A.H, G = A.G;
    const float* w1 = A.params;
    const float* b1 = w1 + H * I;
    const float* w2 = b1 + H;
    const float* b2 = w2 + H * H;
    const float* w3 = b2 + H;
    const float* b3 = w3 + G * H;
    const double wsum = *A.wsum;
    const int64_t ld = A.ld;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < A.E; e += (int64_t)gridDim.x * blockDim.x) {
        float h1[kMaxHidden], h2[kMaxHidden], d2[kMaxHidden];
        for (int j = 0; j < H; ++j) {
            float a = __ldg(&b1[j]);
            for (int i = 0; i < I; ++i) a = __fmaf_rn(__ldg(&w1[j * I + i]), A.feat[(int64_t)i * ld + e], a);
            h1[j] = a > 0.0f ? a : 0.0f;
            A.h1t[(int64_t)j * ld + e] = h1[j];
        }
        for (int j = 0; j < H; ++j) {
            float a = __ldg(&b2[j]);
            for (int i = 0; i < H; ++i) a = __fmaf_rn(__ldg(&w2[j * H + i]), h1[i], a);
            h2[j] = a > 0.0f ? a : 0.0f;
            A.h2t[(int64_t)j * ld + e] = h2[j];
            d2[j] = 0.0f;
        }
        // logits of the present outputs (stored in dz), their maximum
        float m = -INFINITY;
        for (int g = 0; g < G; ++g) {
            const float p = A.target[(int64_t)g * ld + e];
            float z = 0.0f;
            if (p >= 0.0f) {
                z = __ldg(&b3[g]);
                for (int i = 0; i < H; ++i) z = __fmaf_rn(__ldg(&w3[g * H + i]), h2[i], z);
                m = fmaxf(m, z);
            }
            A.dzt[(int64_t)g * ld + e] = z;
        }
        float S = 0.0f, sp = 0.0f, spz = 0.0f;
        for (int g = 0; g < G; ++g) {
            const float p = A.target[(int64_t)g * ld + e];
            if (p < 0.0f) continue;
            const float z = A.dzt[(int64_t)g * ld + e];
            S += expf(z - m);
            sp += p;
            spz = __fmaf_rn(p, z, spz);
        }
        const float om = wsum > 0.0 ? (float)((double)A.weight[e] / wsum) : 0.0f;
        A.lossv[e] = S > 0.0f ? om * (sp * (m + logf(S)) - spz) : 0.0f;
        for (int g = 0; g < G; ++g) {
            const float p = A.target[(int64_t)g * ld + e];
            float dz = 0.0f;
            if (p >= 0.0f && S > 0.0f) {
                const float q = expf(A.dzt[(int64_t)g * ld + e] - m) / S;
                dz = om * (sp * q - p);
                for (int i = 0; i < H; ++i) d2[i] = __fmaf_rn(__ldg(&w3[g * H + i]), dz, d2[i]);
            }
            A.dzt[(int64_t)g * ld + e] = dz;
        }
        for (int j = 0; j < H; ++j) {
            if (!(h2[j] > 0.0f)) d2[j] = 0.0f;
            A.d2t[(int64_t)j * ld + e] = d2[j];
        }
        for (int i = 0; i < H; ++i) {
            float a = 0.0f;
            for (int j = 0; j < H; ++j) a = __fmaf_rn(__ldg(&w2[j * H + i]), d2[j], a);
            A.d1t[(int64_t)i * ld + e] = h1[i] > 0.0f ? a : 0.0f;
        }
    }
}

// C[m][n] = sum_e A[m][e] B[n][e] (B null: 1) for m < M, n < N over e < E,
// rows of length ld.  A 16 x 16 tile of C per CTA, events in chunks of 64
// through shared memory; each chunk's dot product is added to the running
// sum in event order.
__global__ void __launch_bounds__(256) k_learn_abt(const float* __restrict__ Am, const float* __restrict__ Bm, int M,
                                                  int N, int64_t E, int64_t ld, float* __restrict__ C)
{
    __shared__ float As[16][65], Bs[16][65];
    const int tm = threadIdx.x >> 4, tn = threadIdx.x & 15;
    const int m0 = blockIdx.y * 16, n0 = blockIdx.x * 16;
    float acc = 0.0f;
    for (int64_t e0 = 0; e0 < E; e0 += 64) {
        for (int q = threadIdx.x; q < 16 * 64; q += 256) {
            const int r = q >> 6, c = q & 63;
            const int64_t e = e0 + c;
            As[r][c] = (m0 + r < M && e < E) ? Am[(int64_t)(m0 + r) * ld + e] : 0.0f;
            Bs[r][c] = (n0 + r < N && e < E) ? (Bm ? Bm[(int64_t)(n0 + r) * ld + e] : 1.0f) : 0.0f;
        }
        __syncthreads();
        float part = 0.0f;
#pragma unroll 16
        for (int c = 0; c < 64; ++c) part = __fmaf_rn(As[tm][c], Bs[tn][c], part);
        acc += part;
        __syncthreads();
    }
    if (m0 + tm < M && n0 + tn < N) C[(int64_t)(m0 + tm) * N + n0 + tn] = acc;
}

__global__ void k_learn_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                             float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                             float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ---------------------------------------------------------------------------
// Tensor-core training (the network of QMC_PROPOSAL_LEARNED_TC).
// ---------------------------------------------------------------------------
constexpr int kTcTrainWarps = 4;

struct TcTrain {
    TcLayout L;
    int ldt2, ldt3;          // row lengths of W2^T [H][H + 8] and W3^T [H][Gp + 8]
    int o_w2t, o_w3t, bytes;
};

__host__ __device__ inline TcTrain tc_train(int I, int H, int G)
{
    TcTrain T;
    T.L = tc_layout(I, H, G);
    T.ldt2 = H + 8;
    T.ldt3 = T.L.Gp + 8;
    T.o_w2t = T.L.bytes;
    T.o_w3t = T.o_w2t + 2 * H * T.ldt2;
    T.bytes = (T.o_w3t + 2 * H * T.ldt3 + 15) / 16 * 16;
    return T;
}

// W2^T and W3^T (bf16) after the inference layout.
__global__ void k_learn_tc_transpose(const float* __restrict__ prm, TcTrain T, uint8_t* __restrict__ out)
{
    const int I = T.L.I, H = T.L.H, G = T.L.G;
    const float* w2 = prm + H * I + H;
    const float* w3 = w2 + H * H + H;
    __nv_bfloat16* w2t = (__nv_bfloat16*)(out + T.o_w2t);
    __nv_bfloat16* w3t = (__nv_bfloat16*)(out + T.o_w3t);
    const int n2 = H * T.ldt2, n3 = H * T.ldt3;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n2 + n3; e += gridDim.x * blockDim.x) {
        if (e < n2) {
            const int i = e / T.ldt2, j = e % T.ldt2;   // W2^T[i][j] = W2[j][i]
            w2t[e] = __float2bfloat16_rn(j < H ? w2[j * H + i] : 0.0f);
        } else {
            const int f = e - n2, h = f / T.ldt3, g = f % T.ldt3;   // W3^T[h][g] = W3[g][h]
            w3t[f] = __float2bfloat16_rn(g < G ? w3[g * H + h] : 0.0f);
        }
    }
}

// Write a 16-row fragment tile (rows = events, cols = features: C layout
// pairs) to the warp's transpose buffer tr[col][16], as bf16.
__device__ __forceinline__ void tr_put(__nv_bfloat16* tr, int col, int row, float v)
{
    tr[col * 16 + row] = __float2bfloat16_rn(v);
}

// Copy rows [0, F) of the transpose buffer to out[f * ldp + e0 .. e0 + 15].
__device__ __forceinline__ void tr_store(const __nv_bfloat16* tr, int F, uint16_t* out, int64_t ldp, int64_t e0,
                                         int lane)
{
    __syncwarp();
    for (int f = lane; f < F; f += 32) {
        const uint4* src = (const uint4*)(tr + f * 16);
        uint4* dst = (uint4*)(out + (int64_t)f * ldp + e0);
        dst[0] = src[0];
        dst[1] = src[1];
    }
    __syncwarp();
}

// One warp per 16 events: forward pass (bf16 x bf16 -> fp32, GELU), masked
// softmax cross-entropy against the heat-bath shares, dz = w (sum p) q - w p
// (unnormalised: the weight sum divides at the end), then dh2 = dz W3,
// da2 = dh2 gelu'(a2), dh1 = da2 W2, da1 = dh1 gelu'(a1).  Stores h1, h2,
// da1, da2, dz as bf16 rows over events and w CE per event.
__global__ void __launch_bounds__(kTcTrainWarps * 32) k_learn_tc_fwdbwd(LearnTc A)
{
    extern __shared__ __align__(16) uint8_t tsm[];
    const TcTrain T = tc_train(A.I, A.H, A.G);
    const TcLayout& L = T.L;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane >> 2, q = lane & 3;
    for (int i = threadIdx.x; i < T.bytes / 16; i += blockDim.x) ((uint4*)tsm)[i] = ((const uint4*)A.wts)[i];
    const int Gk = (L.Gp + 15) / 16 * 16;   // outputs padded to whole k tiles (zero rows of W3^T, zero dz)
    const int ldo = Gk + 4;
    float* lg = (float*)(tsm + T.bytes) + warp * 16 * ldo;
    const int trrows = L.Gp > L.H ? L.Gp : L.H;
    __nv_bfloat16* tr = (__nv_bfloat16*)((float*)(tsm + T.bytes) + kTcTrainWarps * 16 * ldo) + warp * trrows * 16;
    __syncthreads();
    const __nv_bfloat16* W1 = (const __nv_bfloat16*)(tsm + L.o_w1);
    const __nv_bfloat16* W2 = (const __nv_bfloat16*)(tsm + L.o_w2);
    const __nv_bfloat16* W3 = (const __nv_bfloat16*)(tsm + L.o_w3);
    const __nv_bfloat16* W2T = (const __nv_bfloat16*)(tsm + T.o_w2t);
    const __nv_bfloat16* W3T = (const __nv_bfloat16*)(tsm + T.o_w3t);
    const float* b1 = (const float*)(tsm + L.o_b1);
    const float* b2 = (const float*)(tsm + L.o_b2);
    const float* b3 = (const float*)(tsm + L.o_b3);
    const int H = L.H, G = L.G, I = L.I;
    const int nth = H / 8, kth = H / 16;
    const int64_t ntiles = (A.E + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * kTcTrainWarps + warp; tile < ntiles;
         tile += (int64_t)gridDim.x * kTcTrainWarps) {
        const int64_t e0 = tile * 16;
        const int64_t ea = e0 + grp, eb = e0 + grp + 8;
        auto X = [&](int64_t e, int c) -> float { return (e < A.E && c < I) ? A.feat[(int64_t)c * A.ld + e] : 0.0f; };
        float a1[8][4], a2[8][4];
        uint32_t h[4][4];
        // layer 1
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c = nt * 8 + 2 * q;
            a1[nt][0] = nt < nth ? b1[c] : 0.0f;
            a1[nt][1] = nt < nth ? b1[c + 1] : 0.0f;
            a1[nt][2] = a1[nt][0];
            a1[nt][3] = a1[nt][1];
        }
        for (int kt = 0; kt < L.Ip / 16; ++kt) {
            const int c = kt * 16 + 2 * q;
            uint32_t f[4];
            f[0] = bf16x2(X(ea, c), X(ea, c + 1));
            f[1] = bf16x2(X(eb, c), X(eb, c + 1));
            f[2] = bf16x2(X(ea, c + 8), X(ea, c + 9));
            f[3] = bf16x2(X(eb, c + 8), X(eb, c + 9));
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                if (nt >= nth) break;
                const uint32_t* row = (const uint32_t*)(W1 + (nt * 8 + grp) * L.ld1 + kt * 16 + 2 * q);
                mma_bf16(a1[nt], f, row[0], row[4]);
            }
        }
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            h[kt][0] = bf16x2(tc_gelu(a1[2 * kt][0]), tc_gelu(a1[2 * kt][1]));
            h[kt][1] = bf16x2(tc_gelu(a1[2 * kt][2]), tc_gelu(a1[2 * kt][3]));
            h[kt][2] = bf16x2(tc_gelu(a1[2 * kt + 1][0]), tc_gelu(a1[2 * kt + 1][1]));
            h[kt][3] = bf16x2(tc_gelu(a1[2 * kt + 1][2]), tc_gelu(a1[2 * kt + 1][3]));
        }
        // h1 out (rows = hidden units)
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            if (kt >= kth) break;
            const int c = kt * 16 + 2 * q;
            const __nv_bfloat162* p0 = (const __nv_bfloat162*)&h[kt][0];
            const __nv_bfloat162* p1 = (const __nv_bfloat162*)&h[kt][1];
            const __nv_bfloat162* p2 = (const __nv_bfloat162*)&h[kt][2];
            const __nv_bfloat162* p3 = (const __nv_bfloat162*)&h[kt][3];
            tr[c * 16 + grp] = p0->x;
            tr[(c + 1) * 16 + grp] = p0->y;
            tr[c * 16 + grp + 8] = p1->x;
            tr[(c + 1) * 16 + grp + 8] = p1->y;
            tr[(c + 8) * 16 + grp] = p2->x;
            tr[(c + 9) * 16 + grp] = p2->y;
            tr[(c + 8) * 16 + grp + 8] = p3->x;
            tr[(c + 9) * 16 + grp + 8] = p3->y;
        }
        tr_store(tr, H, A.h1t, A.ldp, e0, lane);
        // layer 2
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c = nt * 8 + 2 * q;
            a2[nt][0] = nt < nth ? b2[c] : 0.0f;
            a2[nt][1] = nt < nth ? b2[c + 1] : 0.0f;
            a2[nt][2] = a2[nt][0];
            a2[nt][3] = a2[nt][1];
        }
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            if (kt >= kth) break;
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                if (nt >= nth) break;
                const uint32_t* row = (const uint32_t*)(W2 + (nt * 8 + grp) * L.ld2 + kt * 16 + 2 * q);
                mma_bf16(a2[nt], h[kt], row[0], row[4]);
            }
        }
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            h[kt][0] = bf16x2(tc_gelu(a2[2 * kt][0]), tc_gelu(a2[2 * kt][1]));
            h[kt][1] = bf16x2(tc_gelu(a2[2 * kt][2]), tc_gelu(a2[2 * kt][3]));
            h[kt][2] = bf16x2(tc_gelu(a2[2 * kt + 1][0]), tc_gelu(a2[2 * kt + 1][1]));
            h[kt][3] = bf16x2(tc_gelu(a2[2 * kt + 1][2]), tc_gelu(a2[2 * kt + 1][3]));
        }
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            if (kt >= kth) break;
            const int c = kt * 16 + 2 * q;
            const __nv_bfloat162* p0 = (const __nv_bfloat162*)&h[kt][0];
            const __nv_bfloat162* p1 = (const __nv_bfloat162*)&h[kt][1];
            const __nv_bfloat162* p2 = (const __nv_bfloat162*)&h[kt][2];
            const __nv_bfloat162* p3 = (const __nv_bfloat162*)&h[kt][3];
            tr[c * 16 + grp] = p0->x;
            tr[(c + 1) * 16 + grp] = p0->y;
            tr[c * 16 + grp + 8] = p1->x;
            tr[(c + 1) * 16 + grp + 8] = p1->y;
            tr[(c + 8) * 16 + grp] = p2->x;
            tr[(c + 9) * 16 + grp] = p2->y;
            tr[(c + 8) * 16 + grp + 8] = p3->x;
            tr[(c + 9) * 16 + grp + 8] = p3->y;
        }
        tr_store(tr, H, A.h2t, A.ldp, e0, lane);
        // layer 3 -> logits
        for (int nt = 0; nt < L.Gp / 8; ++nt) {
            const int c = nt * 8 + 2 * q;
            float d[4] = {b3[c], b3[c + 1], b3[c], b3[c + 1]};
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                if (kt >= kth) break;
                const uint32_t* row = (const uint32_t*)(W3 + (nt * 8 + grp) * L.ld3 + kt * 16 + 2 * q);
                mma_bf16(d, h[kt], row[0], row[4]);
            }
            lg[grp * ldo + c] = d[0];
            lg[grp * ldo + c + 1] = d[1];
            lg[(grp + 8) * ldo + c] = d[2];
            lg[(grp + 8) * ldo + c + 1] = d[3];
        }
        __syncwarp();
        // lanes 0..15: the event's masked softmax, w CE and dz (in place of the logits)
        if (lane < 16) {
            const int64_t e = e0 + lane;
            float* z = lg + lane * ldo;
            float lossw = 0.0f;
            if (e < A.E) {
                const float w = A.weight[e];
                float m = -INFINITY, sp = 0.0f;
                for (int g = 0; g < G; ++g) {
                    const float p = A.target[(int64_t)g * A.ld + e];
                    if (p >= 0.0f) {
                        m = fmaxf(m, z[g]);
                        sp += p;
                    }
                }
                float S = 0.0f;
                for (int g = 0; g < G; ++g)
                    if (A.target[(int64_t)g * A.ld + e] >= 0.0f) S += expf(z[g] - m);
                float ce = 0.0f;
                for (int g = 0; g < Gk; ++g) {
                    const float p = g < G ? A.target[(int64_t)g * A.ld + e] : -1.0f;
                    float dz = 0.0f;
                    if (p >= 0.0f && S > 0.0f) {
                        const float lq = z[g] - m - logf(S);
                        ce -= p * lq;
                        dz = w * (sp * expf(lq) - p);
                    }
                    z[g] = dz;
                }
                lossw = S > 0.0f ? w * ce : 0.0f;
            } else {
                for (int g = 0; g < Gk; ++g) z[g] = 0.0f;
            }
            A.lossv[e] = lossw;
        }
        __syncwarp();
        // dz out (rows = outputs), then dh2 = dz W3 (k over outputs)
        for (int idx = lane; idx < L.Gp * 16; idx += 32) {
            const int g = idx >> 4, r = idx & 15;
            tr[g * 16 + r] = __float2bfloat16_rn(lg[r * ldo + g]);
        }
        tr_store(tr, L.Gp, A.dzt, A.ldp, e0, lane);
        float d2[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) d2[nt][0] = d2[nt][1] = d2[nt][2] = d2[nt][3] = 0.0f;
        for (int kt = 0; kt < Gk / 16; ++kt) {
            const int c = kt * 16 + 2 * q;
            uint32_t f[4];
            f[0] = bf16x2(lg[grp * ldo + c], lg[grp * ldo + c + 1]);
            f[1] = bf16x2(lg[(grp + 8) * ldo + c], lg[(grp + 8) * ldo + c + 1]);
            f[2] = bf16x2(lg[grp * ldo + c + 8], lg[grp * ldo + c + 9]);
            f[3] = bf16x2(lg[(grp + 8) * ldo + c + 8], lg[(grp + 8) * ldo + c + 9]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                if (nt >= nth) break;
                const uint32_t* row = (const uint32_t*)(W3T + (nt * 8 + grp) * T.ldt3 + kt * 16 + 2 * q);
                mma_bf16(d2[nt], f, row[0], row[4]);
            }
        }
        // da2 = dh2 gelu'(a2): out, and as A fragments for dh1 = da2 W2
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            if (nt >= nth) break;
#pragma unroll
            for (int u = 0; u < 4; ++u) d2[nt][u] *= tc_gelu_prime(a2[nt][u]);
            const int c = nt * 8 + 2 * q;
            tr_put(tr, c, grp, d2[nt][0]);
            tr_put(tr, c + 1, grp, d2[nt][1]);
            tr_put(tr, c, grp + 8, d2[nt][2]);
            tr_put(tr, c + 1, grp + 8, d2[nt][3]);
        }
        tr_store(tr, H, A.d2t, A.ldp, e0, lane);
        float d1[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) d1[nt][0] = d1[nt][1] = d1[nt][2] = d1[nt][3] = 0.0f;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            if (kt >= kth) break;
            uint32_t f[4];
            f[0] = bf16x2(d2[2 * kt][0], d2[2 * kt][1]);
            f[1] = bf16x2(d2[2 * kt][2], d2[2 * kt][3]);
            f[2] = bf16x2(d2[2 * kt + 1][0], d2[2 * kt + 1][1]);
            f[3] = bf16x2(d2[2 * kt + 1][2], d2[2 * kt + 1][3]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                if (nt >= nth) break;
                const uint32_t* row = (const uint32_t*)(W2T + (nt * 8 + grp) * T.ldt2 + kt * 16 + 2 * q);
                mma_bf16(d1[nt], f, row[0], row[4]);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            if (nt >= nth) break;
            const int c = nt * 8 + 2 * q;
            tr_put(tr, c, grp, d1[nt][0] * tc_gelu_prime(a1[nt][0]));
            tr_put(tr, c + 1, grp, d1[nt][1] * tc_gelu_prime(a1[nt][1]));
            tr_put(tr, c, grp + 8, d1[nt][2] * tc_gelu_prime(a1[nt][2]));
            tr_put(tr, c + 1, grp + 8, d1[nt][3] * tc_gelu_prime(a1[nt][3]));
        }
        tr_store(tr, H, A.d1t, A.ldp, e0, lane);
    }
}

// Partial weight gradients over one chunk of events (blockIdx.x) for one
// matrix (blockIdx.y: 0 W1 = da1 X^T, 1 W2 = da2 h1^T, 2 W3 = dz h2^T) and
// the bias row sums: bf16 products, fp32 accumulation in event order within
// the chunk.  Output rows of 16 per warp (round robin), every 8-column tile.
__global__ void __launch_bounds__(256) k_learn_tc_wgrad(LearnTc A)
{
    const int I = A.I, H = A.H, G = A.G;
    const TcLayout L = tc_layout(I, H, G);
    const int mat = blockIdx.y;
    const uint16_t* Am = mat == 0 ? A.d1t : (mat == 1 ? A.d2t : A.dzt);
    const uint16_t* Bm = mat == 1 ? A.h1t : A.h2t;   // mat 0 takes the fp32 features
    const int M = mat == 2 ? L.Gp : H;
    const int Mvalid = mat == 2 ? G : H;
    const int N = mat == 0 ? L.Ip : H;
    const int Nvalid = mat == 0 ? I : H;
    const int64_t w_off = mat == 0 ? 0 : (mat == 1 ? (int64_t)H * I + H : (int64_t)H * I + H + H * H + H);
    const int64_t b_off = w_off + (int64_t)Mvalid * Nvalid;
    const int64_t np = (int64_t)H * I + H + H * H + H + (int64_t)G * H + G;
    float* out = A.partials + (int64_t)blockIdx.x * np;
    const int64_t c0 = (int64_t)blockIdx.x * kLearnTcChunk;
    const int64_t c1 = min(A.E, c0 + kLearnTcChunk);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane >> 2, q = lane & 3;
    const int nnt = N / 8;
    for (int mt = warp; mt < (M + 15) / 16; mt += 8) {
        float acc[10][4];
#pragma unroll
        for (int nt = 0; nt < 10; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
        const int ra = mt * 16 + grp, rb = ra + 8;   // rows past M (outputs padded to 8) read as zero
        for (int64_t e0 = c0; e0 < c1; e0 += 16) {
            const uint32_t* ar0 = (const uint32_t*)(Am + (int64_t)ra * A.ldp + e0 + 2 * q);
            const uint32_t* ar1 = (const uint32_t*)(Am + (int64_t)rb * A.ldp + e0 + 2 * q);
            const uint32_t a[4] = {ra < M ? ar0[0] : 0u, rb < M ? ar1[0] : 0u, ra < M ? ar0[4] : 0u,
                                   rb < M ? ar1[4] : 0u};
#pragma unroll
            for (int nt = 0; nt < 10; ++nt) {
                if (nt >= nnt) break;
                const int col = nt * 8 + grp;
                uint32_t b0, b1;
                if (mat == 0) {
                    auto X = [&](int64_t e) -> float {
                        return (col < I && e < A.E) ? A.feat[(int64_t)col * A.ld + e] : 0.0f;
                    };
                    b0 = bf16x2(X(e0 + 2 * q), X(e0 + 2 * q + 1));
                    b1 = bf16x2(X(e0 + 2 * q + 8), X(e0 + 2 * q + 9));
                } else {
                    const uint32_t* br = (const uint32_t*)(Bm + (int64_t)col * A.ldp + e0 + 2 * q);
                    b0 = br[0];
                    b1 = br[4];
                }
                mma_bf16(acc[nt], a, b0, b1);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 10; ++nt) {
            if (nt >= nnt) break;
            const int col = nt * 8 + 2 * q;
            const int r0 = mt * 16 + grp, r1 = r0 + 8;
            if (r0 < Mvalid && col < Nvalid) out[w_off + (int64_t)r0 * Nvalid + col] = acc[nt][0];
            if (r0 < Mvalid && col + 1 < Nvalid) out[w_off + (int64_t)r0 * Nvalid + col + 1] = acc[nt][1];
            if (r1 < Mvalid && col < Nvalid) out[w_off + (int64_t)r1 * Nvalid + col] = acc[nt][2];
            if (r1 < Mvalid && col + 1 < Nvalid) out[w_off + (int64_t)r1 * Nvalid + col + 1] = acc[nt][3];
        }
    }
    // bias: row sums of the signal over the chunk (one thread per row, event order)
    for (int r = threadIdx.x; r < Mvalid; r += blockDim.x) {
        float s = 0.0f;
        const __nv_bfloat16* row = (const __nv_bfloat16*)(Am + (int64_t)r * A.ldp);
        for (int64_t e = c0; e < c1; ++e) s += __bfloat162float(row[e]);
        out[b_off + r] = s;
    }
}

// grad[p] = (sum over chunks of partials[c][p]) / sum of the weights, chunks in order.
__global__ void k_learn_tc_reduce(const float* __restrict__ partials, int64_t nchunks, int64_t np,
                                  const double* __restrict__ wsum, float* __restrict__ grad)
{
    const double ws = *wsum;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t c = 0; c < nchunks; ++c) s += (double)partials[c * np + p];
        grad[p] = ws > 0.0 ? (float)(s / ws) : 0.0f;
    }
}

__global__ void k_learn_tc_scale(double* loss, const double* wsum)
{
    *loss = *wsum > 0.0 ? *loss / *wsum : 0.0;
}

int grid_for(int64_t n, int threads)
{
    const int64_t b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

} // namespace

void launch_learn_events(const LearnArgs& A, cudaStream_t stream)
{
    k_learn_events<<<grid_for(A.max_events, kLearnThreads), kLearnThreads, 0, stream>>>(A);
}

void launch_learn_grad(const LearnGrad& A, float* grad, double* loss, cudaStream_t stream)
{
    const int I = A.I, H = A.H, G = A.G;
    k_learn_sum<<<1, 1024, 0, stream>>>(A.weight, nullptr, A.E, A.wsum);
    k_learn_fwdbwd<<<grid_for(A.E, kLearnThreads), kLearnThreads, 0, stream>>>(A);
    float* gw1 = grad;
    float* gb1 = gw1 + H * I;
    float* gw2 = gb1 + H;
    float* gb2 = gw2 + H * H;
    float* gw3 = gb2 + H;
    float* gb3 = gw3 + G * H;
    auto abt = [&](const float* a, const float* b, int M, int N, float* c) {
        k_learn_abt<<<dim3((N + 15) / 16, (M + 15) / 16), 256, 0, stream>>>(a, b, M, N, A.E, A.ld, c);
    };
    abt(A.d1t, A.feat, H, I, gw1);
    abt(A.d1t, nullptr, H, 1, gb1);
    abt(A.d2t, A.h1t, H, H, gw2);
    abt(A.d2t, nullptr, H, 1, gb2);
    abt(A.dzt, A.h2t, G, H, gw3);
    abt(A.dzt, nullptr, G, 1, gb3);
    k_learn_sum<<<1, 1024, 0, stream>>>(A.lossv, nullptr, A.E, loss);
}

int64_t learn_tc_weights_bytes(int I, int H, int G) { return tc_train(I, H, G).bytes; }

int64_t learn_tc_scratch_bytes(int I, int H, int G, int64_t E)
{
    const TcLayout L = tc_layout(I, H, G);
    const int64_t ldp = (E + 15) / 16 * 16;
    const int64_t np = (int64_t)H * I + H + H * H + H + (int64_t)G * H + G;
    const int64_t chunks = (E + kLearnTcChunk - 1) / kLearnTcChunk;
    return 2 * ldp * (4 * (int64_t)H + L.Gp) + 4 * ldp + 4 * chunks * np + 256;
}

void launch_learn_grad_tc(const LearnTc& A, float* grad, double* loss, cudaStream_t stream)
{
    const TcTrain T = tc_train(A.I, A.H, A.G);
    launch_mlp_tc_pack(A.params, T.L, A.wts, stream);
    k_learn_tc_transpose<<<64, 256, 0, stream>>>(A.params, T, A.wts);
    k_learn_sum<<<1, 1024, 0, stream>>>(A.weight, nullptr, A.E, A.wsum);
    const int trrows = T.L.Gp > T.L.H ? T.L.Gp : T.L.H;
    const int Gk = (T.L.Gp + 15) / 16 * 16;
    const int smem = T.bytes + kTcTrainWarps * 16 * (Gk + 4) * 4 + kTcTrainWarps * trrows * 16 * 2;
    static bool attr = false;
    if (!attr) {
        const TcTrain big = tc_train(80, 64, 256);
        cudaFuncSetAttribute(k_learn_tc_fwdbwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             big.bytes + kTcTrainWarps * 16 * (256 + 4) * 4 + kTcTrainWarps * 256 * 16 * 2 + 1024);
        attr = true;
    }
    const int64_t ntiles = (A.E + 15) / 16;
    const int blocks = (int)std::min<int64_t>((ntiles + kTcTrainWarps - 1) / kTcTrainWarps, 4096);
    k_learn_tc_fwdbwd<<<blocks > 0 ? blocks : 1, kTcTrainWarps * 32, smem, stream>>>(A);
    const int64_t chunks = (A.E + kLearnTcChunk - 1) / kLearnTcChunk;
    k_learn_tc_wgrad<<<dim3((unsigned)chunks, 3), 256, 0, stream>>>(A);
    const int64_t np = (int64_t)A.H * A.I + A.H + A.H * A.H + A.H + (int64_t)A.G * A.H + A.G;
    k_learn_tc_reduce<<<grid_for(np, 256), 256, 0, stream>>>(A.partials, chunks, np, A.wsum, grad);
    k_learn_sum<<<1, 1024, 0, stream>>>(A.lossv, nullptr, A.E, loss);
    k_learn_tc_scale<<<1, 1, 0, stream>>>(loss, A.wsum);
}

int learn_grad_launch_count() { return 9; }

void launch_learn_adam(float* p, const float* g, float* m, float* v, int64_t n, int64_t t, float lr, float b1,
                       float b2, float eps, cudaStream_t stream)
{
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    k_learn_adam<<<grid_for(n, kLearnThreads), kLearnThreads, 0, stream>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
}

} // namespace qmc
