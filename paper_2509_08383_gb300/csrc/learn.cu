// Training of the learned inverse-square-root stand-in (FP32, hand-written
// kernels): a 1 -> H -> 1 network with square activations,
//   f(u) = b0 + sum_j v_j (w_j u + b_j)^2,   u = (x - mid) / half,
// fitted to 1/sqrt(x) on logged variance inputs x by full-batch Adam (rate
// decayed by a half cosine) on the mean squared relative error
//   L = mean_i (f(u_i) sqrt(x_i) - 1)^2.
// The network is a quadratic in x, so the host collapses it to A x^2 + B x + C,
// which the encrypted circuit evaluates in two levels.
#include <cmath>
#include <cstring>

#include "context.h"

namespace he {

constexpr int NET_H = 16;
constexpr int NET_P = 3 * NET_H + 1;  // w[H], b[H], v[H], b0
constexpr int NET_T = 256;

// full-batch gradient: every block reduces its samples' gradients and adds
// them to g[NET_P] (and the loss to g[NET_P]) with one atomic per parameter
__global__ void __launch_bounds__(NET_T) k_net_grad(const float2 *xs, int n, const float *p, float *g) {
    __shared__ float sp[NET_P];
    __shared__ float red[NET_T / 32][NET_P + 1];
    for (int i = threadIdx.x; i < NET_P; i += blockDim.x) sp[i] = p[i];
    __syncthreads();
    float acc[NET_P + 1];
#pragma unroll
    for (int i = 0; i <= NET_P; i++) acc[i] = 0.f;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const float u = xs[s].x, r = xs[s].y;  // normalised input, sqrt(x)
        float a[NET_H], f = sp[3 * NET_H];
#pragma unroll
        for (int j = 0; j < NET_H; j++) {
            a[j] = fmaf(sp[j], u, sp[NET_H + j]);
            f = fmaf(sp[2 * NET_H + j], a[j] * a[j], f);
        }
        const float e = f * r - 1.f, d = 2.f * e * r;  // dL/df per sample
#pragma unroll
        for (int j = 0; j < NET_H; j++) {
            const float t = 2.f * sp[2 * NET_H + j] * a[j] * d;
            acc[j] += t * u;                  // dw_j
            acc[NET_H + j] += t;              // db_j
            acc[2 * NET_H + j] += a[j] * a[j] * d;  // dv_j
        }
        acc[3 * NET_H] += d;                  // db0
        acc[NET_P] += e * e;                  // loss
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i <= NET_P; i++) {
        float v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= NET_P; i += blockDim.x) {
        float v = 0.f;
        for (int w = 0; w < NET_T / 32; w++) v += red[w][i];
        atomicAdd(&g[i], v);
    }
}

// Adam step on the mean gradient with the rate decayed over the run by a
// half cosine; each thread clears the accumulator words it read (thread 0
// also records and clears the loss)
__global__ void k_net_adam(float *p, float *g, float *m, float *v, int n, float lr0, int step, int steps,
                           float *loss_out) {
    const float lr = lr0 * 0.5f * (1.f + cospif((float)step / (float)steps));
    const int i = threadIdx.x;
    if (i == 0) {
        loss_out[0] = g[NET_P] / (float)n;
        g[NET_P] = 0.f;
    }
    if (i < NET_P) {
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float gi = g[i] / (float)n;
        m[i] = b1 * m[i] + (1.f - b1) * gi;
        v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
        const float mh = m[i] / (1.f - powf(b1, (float)step)), vh = v[i] / (1.f - powf(b2, (float)step));
        p[i] -= lr * mh / (sqrtf(vh) + eps);
        g[i] = 0.f;
    }
}

// splitmix64, for the initial weights
static u64 splitmix(u64 &s) {
    u64 z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void learn_invsqrt(he_ctx *cx, const float *x_host, size_t n, int steps, float lr, u64 seed, double *abc,
                   double *loss) {
    if (n < 3 || steps < 1) throw Error{HE_EINVAL, "training needs at least 3 samples and 1 step"};
    double lo = x_host[0], hi = x_host[0];
    for (size_t i = 0; i < n; i++) {
        if (!(x_host[i] > 0.f) || !std::isfinite(x_host[i])) throw Error{HE_ERANGE, "variance inputs must be positive"};
        lo = std::min(lo, (double)x_host[i]);
        hi = std::max(hi, (double)x_host[i]);
    }
    const double mid = 0.5 * (lo + hi), half = std::max(0.5 * (hi - lo), 1e-30);
    std::vector<float2> h(n);
    for (size_t i = 0; i < n; i++)
        h[i] = make_float2((float)((x_host[i] - mid) / half), (float)std::sqrt((double)x_host[i]));
    // initial weights: first layer uniform in (-1, 1) (on inputs in [-1, 1]),
    // output weights +-0.1/H alternating in sign, b0 the mean target
    std::vector<float> p(NET_P);
    u64 s = seed;
    double tmean = 0;
    for (size_t i = 0; i < n; i++) tmean += 1.0 / std::sqrt((double)x_host[i]);
    tmean /= (double)n;
    for (int j = 0; j < NET_H; j++) {
        p[j] = (float)(((double)(splitmix(s) >> 11) / 9007199254740992.0 - 0.5) * 2.0);
        p[NET_H + j] = (float)(((double)(splitmix(s) >> 11) / 9007199254740992.0 - 0.5) * 2.0);
        p[2 * NET_H + j] = (float)((j & 1 ? -0.1 : 0.1) / NET_H);
    }
    p[3 * NET_H] = (float)tmean;
    Scratch sc{cx, {}};
    const size_t words = (n * sizeof(float2) + 7) / 8 + 4 * ((NET_P + 2 + 1) / 2 + 1);
    u64 *buf = sc.get(words);
    float2 *d_x = reinterpret_cast<float2 *>(buf);
    float *d_p = reinterpret_cast<float *>(buf + (n * sizeof(float2) + 7) / 8);
    float *d_g = d_p + (NET_P + 2), *d_m = d_g + (NET_P + 2), *d_v = d_m + (NET_P + 2);
    cudaStream_t st = cx->stream;
    check_cuda(cudaMemcpyAsync(d_x, h.data(), n * sizeof(float2), cudaMemcpyHostToDevice, st), "training data");
    check_cuda(cudaMemcpyAsync(d_p, p.data(), NET_P * sizeof(float), cudaMemcpyHostToDevice, st), "weights");
    check_cuda(cudaMemsetAsync(d_g, 0, 3 * (NET_P + 2) * sizeof(float), st), "optimiser state");
    const int blocks = (int)std::min<size_t>(152 * 4, (n + NET_T - 1) / NET_T);
    for (int it = 1; it <= steps; it++) {
        k_net_grad<<<blocks, NET_T, 0, st>>>(d_x, (int)n, d_p, d_g);
        k_net_adam<<<1, 64, 0, st>>>(d_p, d_g, d_m, d_v, (int)n, lr, it, steps, d_m + NET_P + 1);
    }
    float fin[NET_P + 2];
    check_cuda(cudaMemcpyAsync(fin, d_p, NET_P * sizeof(float), cudaMemcpyDeviceToHost, st), "weights");
    check_cuda(cudaMemcpyAsync(&fin[NET_P], d_m + NET_P + 1, sizeof(float), cudaMemcpyDeviceToHost, st), "loss");
    check_cuda(cudaStreamSynchronize(st), "training");
    // collapse: f = b0 + sum v (w (x - mid)/half + b)^2 = A x^2 + B x + C
    double A = 0, B = 0, C = fin[3 * NET_H];
    for (int j = 0; j < NET_H; j++) {
        const double w = fin[j] / half, c0 = fin[NET_H + j] - fin[j] * mid / half, v = fin[2 * NET_H + j];
        A += v * w * w;
        B += 2.0 * v * w * c0;
        C += v * c0 * c0;
    }
    abc[0] = A;
    abc[1] = B;
    abc[2] = C;
    if (loss) *loss = fin[NET_P];
}

}  // namespace he
