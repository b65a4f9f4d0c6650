// mlp.cu -- training of the learned bucket classifier on the GPU: loss and
// gradient (forward and backward written out), Adam, all in one cooperative
// launch; plus the standalone loss/gradient entry point used to check the
// gradients against the CPU oracle.
#include <algorithm>
#include <cooperative_groups.h>

#include "mlp.cuh"

namespace bsps {

constexpr int kMlpThreads = 128;       // one training point per thread per step
constexpr int kMlpMaxPoints = kMlpPointsMax;
constexpr int kMlpSteps = 200;
constexpr float kMlpLr = 1e-2f;

// Per-CTA gradient of the mean squared error over the CTA's points
// [p0, p0+np) (at most kMlpThreads), divided by the global point count m.
// Writes the 1153 partial sums to `part` and returns the partial loss sum.
__device__ float mlp_cta_grad(const float *w, const float *__restrict__ x, const float *__restrict__ y, int64_t p0,
                              int np, int64_t m, float *part, float *scratch) {
    // scratch: h1[kMlpThreads][33], dz2[kMlpThreads][33], dz1[kMlpThreads][33], h2[..][33], xs, dy
    float *sh1 = scratch;
    float *sdz2 = sh1 + kMlpThreads * 33;
    float *sdz1 = sdz2 + kMlpThreads * 33;
    float *sh2 = sdz1 + kMlpThreads * 33;
    float *sx = sh2 + kMlpThreads * 33;
    float *sdy = sx + kMlpThreads;
    float *sloss = sdy + kMlpThreads;
    const int t = threadIdx.x;
    float lossp = 0.0f;
    if (t < np) {
        const float xi = x[p0 + t];
        float z1[kH], h1[kH], z2[kH];
#pragma unroll
        for (int j = 0; j < kH; ++j) {
            z1[j] = fmaf(w[kW1 + j], xi, w[kB1 + j]);
            h1[j] = fmaxf(z1[j], 0.0f);
        }
        float out = w[kB3];
        for (int i = 0; i < kH; ++i) {
            float z = w[kB2 + i];
#pragma unroll
            for (int j = 0; j < kH; ++j) z = fmaf(w[kW2 + i * kH + j], h1[j], z);
            z2[i] = z;
            out = fmaf(w[kW3 + i], fmaxf(z, 0.0f), out);
        }
        const float r = out - y[p0 + t];
        lossp = r * r;
        const float dy = 2.0f * r / (float)m;
        float dz1[kH];
#pragma unroll
        for (int j = 0; j < kH; ++j) dz1[j] = 0.0f;
        for (int i = 0; i < kH; ++i) {
            const float d2 = z2[i] > 0.0f ? dy * w[kW3 + i] : 0.0f;
            sdz2[t * 33 + i] = d2;
            sh2[t * 33 + i] = fmaxf(z2[i], 0.0f);
#pragma unroll
            for (int j = 0; j < kH; ++j) dz1[j] = fmaf(d2, w[kW2 + i * kH + j], dz1[j]);
        }
#pragma unroll
        for (int j = 0; j < kH; ++j) {
            sh1[t * 33 + j] = h1[j];
            sdz1[t * 33 + j] = z1[j] > 0.0f ? dz1[j] : 0.0f;
        }
        sx[t] = xi;
        sdy[t] = dy;
    }
    __syncthreads();
    // sums over the CTA's points, one or more parameters per thread
    for (int k = t; k < kParams; k += kMlpThreads) {
        float g = 0.0f;
        if (k < kB1) {                     // W1[j] = sum dz1[j] * x
            for (int p = 0; p < np; ++p) g = fmaf(sdz1[p * 33 + k], sx[p], g);
        } else if (k < kW2) {              // b1[j] = sum dz1[j]
            for (int p = 0; p < np; ++p) g += sdz1[p * 33 + (k - kB1)];
        } else if (k < kB2) {              // W2[i][j] = sum dz2[i] * h1[j]
            const int i = (k - kW2) / kH, j = (k - kW2) % kH;
            for (int p = 0; p < np; ++p) g = fmaf(sdz2[p * 33 + i], sh1[p * 33 + j], g);
        } else if (k < kW3) {              // b2[i] = sum dz2[i]
            for (int p = 0; p < np; ++p) g += sdz2[p * 33 + (k - kB2)];
        } else if (k < kB3) {              // w3[i] = sum dy * h2[i]
            for (int p = 0; p < np; ++p) g = fmaf(sdy[p], sh2[p * 33 + (k - kW3)], g);
        } else {                           // b3 = sum dy
            for (int p = 0; p < np; ++p) g += sdy[p];
        }
        part[k] = g;
    }
    // partial loss
    float l = lossp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((t & 31) == 0) sloss[t >> 5] = l;
    __syncthreads();
    float tot = 0.0f;
    for (int i = 0; i < kMlpThreads / 32; ++i) tot += sloss[i];
    __syncthreads();
    return tot;
}

constexpr int kMlpScratchFloats = 4 * kMlpThreads * 33 + 2 * kMlpThreads + 8;

struct MlpTrainArgs {
    float *params;        // kParams, trained in place
    float *m, *v;         // Adam moments
    float *part;          // grid * (kParams + 1) partial gradients (+ partial loss)
    const float *x, *y;   // training points
    const int64_t *npts;  // number of training points (device)
    int steps;
    float lr;
    float *loss_first, *loss_last;  // nullable
};

// All training steps in one cooperative launch: every CTA computes the
// gradient of its points, the grid synchronises, CTA g reduces and applies
// Adam (Kingma & Ba) to its share of the parameters, the grid synchronises.
__global__ void __launch_bounds__(kMlpThreads) mlp_train_kernel(MlpTrainArgs a) {
    namespace cg = cooperative_groups;
    auto grid = cg::this_grid();
    __shared__ float w[kParams + 3];
    __shared__ float scratch[kMlpScratchFloats];
    __shared__ float red[kMlpThreads / 32];
    const int G = gridDim.x, g = blockIdx.x, t = threadIdx.x;
    const int64_t npts = *a.npts;
    if (npts == 0) return;  // nothing to learn from (uniform across the grid)
    const int64_t per = (npts + G - 1) / G;
    const int64_t p0 = g * per;
    const int np = (int)imax64(0, imin64(per, npts - p0));
    for (int step = 1; step <= a.steps + 1; ++step) {
        for (int k = t; k < kParams; k += kMlpThreads) w[k] = a.params[k];
        __syncthreads();
        float *part = a.part + (int64_t)g * (kParams + 1);
        const float lp = mlp_cta_grad(w, a.x, a.y, p0, np, npts, part, scratch);
        if (t == 0) part[kParams] = lp;
        grid.sync();
        if (step == a.steps + 1) {   // final pass only measures the loss
            if (g == 0) {
                float l = 0.0f;
                for (int c = t; c < G; c += kMlpThreads) l += a.part[(int64_t)c * (kParams + 1) + kParams];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
                if ((t & 31) == 0) red[t >> 5] = l;
                __syncthreads();
                if (t == 0 && a.loss_last) {
                    float s = 0.0f;
                    for (int i = 0; i < kMlpThreads / 32; ++i) s += red[i];
                    *a.loss_last = s / (float)npts;
                }
            }
            break;
        }
        // reduce and update this CTA's parameters
        const float b1c = 1.0f - powf(0.9f, (float)step), b2c = 1.0f - powf(0.999f, (float)step);
        for (int k = g; k < kParams + 1; k += G) {
            float s = 0.0f;
            for (int c = t; c < G; c += kMlpThreads) s += a.part[(int64_t)c * (kParams + 1) + k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if ((t & 31) == 0) red[t >> 5] = s;
            __syncthreads();
            if (t == 0) {
                float gk = 0.0f;
                for (int i = 0; i < kMlpThreads / 32; ++i) gk += red[i];
                if (k == kParams) {
                    if (step == 1 && a.loss_first) *a.loss_first = gk / (float)npts;
                } else {
                    const float mk = 0.9f * a.m[k] + 0.1f * gk;
                    const float vk = 0.999f * a.v[k] + 0.001f * gk * gk;
                    a.m[k] = mk;
                    a.v[k] = vk;
                    a.params[k] -= a.lr * (mk / b1c) / (sqrtf(vk / b2c) + 1e-8f);
                }
            }
            __syncthreads();
        }
        grid.sync();
    }
}

// Loss and gradient only (for the gradient check against the CPU oracle).
__global__ void __launch_bounds__(kMlpThreads) mlp_grad_kernel(const float *params, const float *x, const float *y,
                                                               int64_t m, float *part) {
    __shared__ float w[kParams + 3];
    __shared__ float scratch[kMlpScratchFloats];
    for (int k = threadIdx.x; k < kParams; k += kMlpThreads) w[k] = params[k];
    __syncthreads();
    const int64_t p0 = (int64_t)blockIdx.x * kMlpThreads;
    const int np = (int)imin64(kMlpThreads, m - p0);
    float *pp = part + (int64_t)blockIdx.x * (kParams + 1);
    const float lp = mlp_cta_grad(w, x, y, p0, np, m, pp, scratch);
    if (threadIdx.x == 0) pp[kParams] = lp;
}

__global__ void mlp_grad_reduce_kernel(const float *part, int G, int64_t m, float *grad, float *loss) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > kParams) return;
    float s = 0.0f;
    for (int c = 0; c < G; ++c) s += part[(int64_t)c * (kParams + 1) + k];
    if (k == kParams) {
        if (loss) *loss = s / (float)m;
    } else {
        grad[k] = s;
    }
}

// ---------------------------------------------------------------------------
// Training set from the sorted sample and the initial parameters.
// x_m = normalised value of the sample record of rank r_m (real keys only),
// y_m = (r_m + 1/2) / S, ranks evenly spaced.  Layer-1 kinks start at the
// training points' quantiles; the rest is drawn from Philox with the seed.
// ---------------------------------------------------------------------------
template <int DT>
__global__ void mlp_prepare_kernel(LsdBuffers<typename KeyTraits<DT>::T> b, const int32_t *table, int npos, int64_t S,
                                   int64_t n, MlpNorm *norm, float *x, float *y, int64_t *npts_out) {
    using K = typename KeyTraits<DT>::T;
    const int fin = table[1 + 3 * npos];
    const K *sphi_sorted = b.phi[fin];
    const uint32_t *stag_sorted = b.tag[fin];
    __shared__ int64_t s_real;
    if (threadIdx.x == 0) {
        int64_t lo = 0, hi = S;  // first pad record (tag >= n)
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if ((int64_t)stag_sorted[mid] < n) lo = mid + 1;
            else hi = mid;
        }
        s_real = lo;
        const double vlo = lo > 0 ? key_value<DT>(KeyTraits<DT>::inv(sphi_sorted[0])) : 0.0;
        const double vhi = lo > 0 ? key_value<DT>(KeyTraits<DT>::inv(sphi_sorted[lo - 1])) : 1.0;
        MlpNorm nm;
        nm.lo = vlo;
        nm.lo_f = (float)vlo;
        const double span = vhi - vlo;
        nm.scale = (span > 0 && span < 1e300) ? (float)(1.0 / span) : 0.0f;
        *norm = nm;
        *npts_out = lo < kMlpMaxPoints ? lo : kMlpMaxPoints;
    }
    __syncthreads();
    const int64_t real = s_real;
    const int64_t M = real < kMlpMaxPoints ? real : kMlpMaxPoints;
    const MlpNorm nm = *norm;
    for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
        const int64_t r = M > 1 ? i * (real - 1) / (M - 1) : 0;
        const K bits = KeyTraits<DT>::inv(sphi_sorted[r]);
        float xi = mlp_input<DT>(bits, nm);
        if (!(xi == xi)) xi = 0.0f;
        x[i] = xi;
        y[i] = (float)(((double)r + 0.5) / (double)S);
    }
}

__global__ void mlp_init_kernel(const float *x, const int64_t *npts, uint64_t seed, float *params, float *m,
                                float *v) {
    const int t = threadIdx.x;  // blockDim >= 64
    const int64_t M = *npts;
    // uniform draws from Philox4x64-10, key (seed, 1), counter (t, 0, 0, 0)
    auto unif = [&](int idx) {
        uint64_t c[4] = {(uint64_t)idx, 0, 0, 0};
        philox4x64_10(c, seed, 1);
        return (float)((c[0] >> 40) * (1.0 / 16777216.0));
    };
    __shared__ float q[kH], wmax;
    if (t < kH) q[t] = M > 0 ? x[(int64_t)((t + 0.5) / kH * M)] : (t + 0.5f) / kH;
    __syncthreads();
    if (t == 0) {
        float mx = 0.0f;
        for (int j = 0; j < kH; ++j) {
            const float gap = fmaxf(q[j] - (j ? q[j - 1] : 0.0f), 1e-6f);
            mx = fmaxf(mx, 1.0f / gap);
        }
        wmax = mx;
    }
    __syncthreads();
    if (t < kH) {
        const float gap = fmaxf(q[t] - (t ? q[t - 1] : 0.0f), 1e-6f);
        const float w1 = (1.0f / gap) / wmax * 50.0f;
        params[kW1 + t] = w1;
        params[kB1 + t] = -w1 * q[t];
        params[kB2 + t] = 0.01f;
        const float a3 = sqrtf(6.0f / 33.0f);
        params[kW3 + t] = (2.0f * unif(2048 + t) - 1.0f) * a3;
    }
    const float a2 = 0.5f * sqrtf(6.0f / 64.0f);
    for (int k = t; k < kH * kH; k += blockDim.x) params[kW2 + k] = (2.0f * unif(k) - 1.0f) * a2;
    if (t == 0) params[kB3] = 0.0f;
    for (int k = t; k < kParams; k += blockDim.x) {
        m[k] = 0.0f;
        v[k] = 0.0f;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int mlp_train_grid() {
    static int cached = 0;
    if (cached) return cached;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mlp_train_kernel, kMlpThreads, 0);
    cached = std::max(1, std::min(std::min(sms * std::max(occ, 1), kMlpMaxPoints / kMlpThreads), kMlpGridMax));
    return cached;
}

template <int DT> static cudaError_t launch_mlp_train_t(const Ctx &c) {
    using K = typename KeyTraits<DT>::T;
    const Plan &p = c.pl;
    const int npos = 4 + (int)sizeof(K);
    LsdBuffers<K> b;
    b.phi[0] = (K *)c.ly.sphi[0];
    b.phi[1] = (K *)c.ly.sphi[1];
    b.tag[0] = c.ly.stag[0];
    b.tag[1] = c.ly.stag[1];
    mlp_prepare_kernel<DT><<<1, 256, 0, c.stream>>>(b, c.ly.lsd_table, npos, p.sample_size, p.n, c.ly.mlp_norm,
                                                    c.ly.mlp_x, c.ly.mlp_y, c.ly.mlp_npts);
    mlp_init_kernel<<<1, 256, 0, c.stream>>>(c.ly.mlp_x, c.ly.mlp_npts, p.seed, c.ly.mlp_params, c.ly.mlp_m,
                                             c.ly.mlp_v);
    MlpTrainArgs a;
    a.params = c.ly.mlp_params;
    a.m = c.ly.mlp_m;
    a.v = c.ly.mlp_v;
    a.part = c.ly.mlp_part;
    a.x = c.ly.mlp_x;
    a.y = c.ly.mlp_y;
    a.npts = c.ly.mlp_npts;
    a.steps = kMlpSteps;
    a.lr = kMlpLr;
    a.loss_first = c.dbg.mlp_loss ? c.dbg.mlp_loss : nullptr;
    a.loss_last = c.dbg.mlp_loss ? c.dbg.mlp_loss + 1 : nullptr;
    const int64_t max_pts = std::min<int64_t>(p.sample_size, kMlpMaxPoints);
    const int G = std::max(1, std::min(mlp_train_grid(), (int)((max_pts + kMlpThreads - 1) / kMlpThreads)));
    void *args[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)mlp_train_kernel, dim3(G), dim3(kMlpThreads), args, 0,
                                                c.stream);
    if (e != cudaSuccess) return e;
    if (c.dbg.mlp_params)
        e = cudaMemcpyAsync(c.dbg.mlp_params, c.ly.mlp_params, sizeof(float) * kParams, cudaMemcpyDeviceToDevice,
                            c.stream);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_mlp_train(const Ctx &c) {
    switch (c.pl.dtype) {
    case BSPS_U32: return launch_mlp_train_t<BSPS_U32>(c);
    case BSPS_I32: return launch_mlp_train_t<BSPS_I32>(c);
    case BSPS_F32: return launch_mlp_train_t<BSPS_F32>(c);
    default: return launch_mlp_train_t<BSPS_F64>(c);
    }
}

} // namespace bsps

using namespace bsps;

extern "C" int bsps_mlp_workspace_size(int64_t m, size_t *bytes) {
    if (!bytes || m < 0) return BSPS_ERR_INVALID_ARG;
    const int64_t G = (m + kMlpThreads - 1) / kMlpThreads;
    *bytes = (size_t)std::max<int64_t>(G, 1) * (kParams + 1) * sizeof(float) + 256;
    return BSPS_OK;
}

extern "C" int bsps_mlp_loss_grad(const float *d_params, const float *d_x, const float *d_y, int64_t m, float *d_grad,
                                  float *d_loss, void *d_ws, size_t ws_bytes, void *stream) {
    if (m <= 0 || !d_params || !d_x || !d_y || !d_grad) return BSPS_ERR_INVALID_ARG;
    size_t need = 0;
    bsps_mlp_workspace_size(m, &need);
    if (!d_ws || ws_bytes < need) return BSPS_ERR_WORKSPACE_TOO_SMALL;
    const int G = (int)((m + kMlpThreads - 1) / kMlpThreads);
    cudaStream_t s = (cudaStream_t)stream;
    mlp_grad_kernel<<<G, kMlpThreads, 0, s>>>(d_params, d_x, d_y, m, (float *)d_ws);
    mlp_grad_reduce_kernel<<<(kParams + 1 + 255) / 256, 256, 0, s>>>((const float *)d_ws, G, m, d_grad, d_loss);
    return cudaGetLastError() == cudaSuccess ? BSPS_OK : BSPS_ERR_CUDA;
}
