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
#include <math.h>
#include <stdint.h>

#include "column_eval.h"
#include "kernels.h"

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

int learn_grad_launch_count() { return 9; }

void launch_learn_adam(float* p, const float* g, float* m, float* v, int64_t n, int64_t t, float lr, float b1,
                       float b2, float eps, cudaStream_t stream)
{
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    k_learn_adam<<<grid_for(n, kLearnThreads), kLearnThreads, 0, stream>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
}

} // namespace qmc
