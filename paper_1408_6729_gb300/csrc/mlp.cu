// mlp.cu -- training of the learned bucket classifier on the GPU: the training
// set from the sorted sample, the spline start, the layer-2 features of every
// training point, and full-batch gradient steps on the output layer; plus the
// loss and gradient of the whole network (forward and backward written out)
// behind the entry point that checks them against the CPU oracle.
#include <algorithm>

#include "mlp.cuh"

namespace bsps {

constexpr int kMlpThreads = 128;       // one training point per thread per step
constexpr int kMlpMaxPoints = kMlpPointsMax;
constexpr int kMlpSteps = 16;          // gradient steps from the spline start
// Full-batch gradient descent on the output layer (w3, b3): the loss is a
// convex quadratic there with Hessian 2 E[h h^T], h = (h2, 1), whose largest
// eigenvalue is at most 2 * 33 for inputs in [0, 1]; a step below 2/66
// lowers the loss at every step.
constexpr float kMlpLr = 0.02f;
constexpr int kMlpTrainPoints = 4096;  // training points drawn from the sorted sample

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

// Layers 1 and 2 stay at their start; their output for every training point
// is computed once.  h2 holds kH x npts floats (feature-major, so that the
// training steps read consecutive points).
__global__ void __launch_bounds__(kMlpThreads) mlp_features_kernel(const float *params, const float *x,
                                                                  const int64_t *npts, float *h2) {
    __shared__ float w[kParams + 3];
    for (int k = threadIdx.x; k < kParams; k += kMlpThreads) w[k] = params[k];
    __syncthreads();
    const int64_t m = *npts;
    for (int64_t p = (int64_t)blockIdx.x * kMlpThreads + threadIdx.x; p < m; p += (int64_t)gridDim.x * kMlpThreads) {
        const float xi = x[p];
        float h1[kH];
#pragma unroll
        for (int j = 0; j < kH; ++j) h1[j] = fmaxf(fmaf(w[kW1 + j], xi, w[kB1 + j]), 0.0f);
        for (int i = 0; i < kH; ++i) {
            float z = w[kB2 + i];
#pragma unroll
            for (int j = 0; j < kH; ++j) z = fmaf(w[kW2 + i * kH + j], h1[j], z);
            h2[(int64_t)i * m + p] = fmaxf(z, 0.0f);
        }
    }
}

// Full-batch gradient descent on the output layer (w3, b3) from the cached
// features, one CTA: every step sums 2 r h2 / m and 2 r / m over the points
// (r = y - target) and moves w3, b3 against them.  Records the loss before the
// first step and after the last.
constexpr int kMlpHeadThreads = 1024;
__global__ void __launch_bounds__(kMlpHeadThreads) mlp_head_kernel(float *params, const float *h2, const float *y,
                                                                   const int64_t *npts, int steps, float lr,
                                                                   float *loss_first, float *loss_last) {
    constexpr int W = kMlpHeadThreads / 32, NV = kH + 2;  // w3 gradient, b3 gradient, loss
    __shared__ float head[kH + 1];
    __shared__ float part[W][NV];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t m = *npts;
    if (m == 0) return;
    if (t <= kH) head[t] = params[kW3 + t];  // w3[0..31], b3
    __syncthreads();
    for (int step = 0; step <= steps; ++step) {
        float g[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) g[i] = 0.0f;
        for (int64_t p = t; p < m; p += kMlpHeadThreads) {
            float f[kH];
#pragma unroll
            for (int i = 0; i < kH; ++i) f[i] = h2[(int64_t)i * m + p];
            float out = head[kH];
#pragma unroll
            for (int i = 0; i < kH; ++i) out = fmaf(head[i], f[i], out);
            const float r = out - y[p];
            const float dy = 2.0f * r / (float)m;
#pragma unroll
            for (int i = 0; i < kH; ++i) g[i] = fmaf(dy, f[i], g[i]);
            g[kH] += dy;
            g[kH + 1] = fmaf(r, r, g[kH + 1]);
        }
#pragma unroll
        for (int i = 0; i < NV; ++i) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) g[i] += __shfl_xor_sync(0xffffffffu, g[i], o);
        }
        if (lane == 0)
#pragma unroll
            for (int i = 0; i < NV; ++i) part[warp][i] = g[i];
        __syncthreads();
        if (t < NV) {
            float tot = 0.0f;
            for (int q = 0; q < W; ++q) tot += part[q][t];
            if (t == kH + 1) {
                if (step == 0 && loss_first) *loss_first = tot / (float)m;
                if (step == steps && loss_last) *loss_last = tot / (float)m;
            } else if (step < steps) {
                head[t] -= lr * tot;  // t < kH: w3[t]; t == kH: b3
            }
        }
        __syncthreads();
    }
    if (t <= kH) params[kW3 + t] = head[t];
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
// y_m = (r_m + 1/2) / S, ranks evenly spaced.
//
// Start: the network is set to the piecewise-linear interpolant of the
// training points at 33 knots of evenly spaced rank (equal x merged): unit j
// of layer 1 is relu(x - knot_j), layer 2 passes its input through
// (W2 = I, b2 = 0; relu is the identity on relu outputs), and the output
// weights are the slope changes at the knots.  Training then refines it.
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
        *npts_out = lo < kMlpTrainPoints ? lo : kMlpTrainPoints;
    }
    __syncthreads();
    const int64_t real = s_real;
    const int64_t M = real < kMlpTrainPoints ? real : kMlpTrainPoints;
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

__global__ void mlp_init_kernel(const float *x, const float *y, const int64_t *npts, float *params) {
    const int t = threadIdx.x;  // blockDim >= kH
    const int64_t M = *npts;
    __shared__ float kx[kH + 1], ky[kH + 1];
    __shared__ int nk;
    if (t == 0) {
        int c = 0;
        for (int j = 0; j <= kH && M > 0; ++j) {
            const int64_t i = M > 1 ? (int64_t)j * (M - 1) / kH : 0;
            const float xv = x[i], yv = y[i];
            if (c == 0 || xv > kx[c - 1]) {
                kx[c] = xv;
                ky[c] = yv;
                ++c;
            } else {
                ky[c - 1] = yv;  // equal x: one knot
            }
        }
        nk = c;
    }
    __syncthreads();
    const int segs = nk > 1 ? nk - 1 : 0;
    auto slope = [&](int j) { return (ky[j + 1] - ky[j]) / (kx[j + 1] - kx[j]); };
    if (t < kH) {
        const bool on = t < segs;
        params[kW1 + t] = on ? 1.0f : 0.0f;
        params[kB1 + t] = on ? -kx[t] : -1.0f;  // unused units stay at zero
        params[kB2 + t] = 0.0f;
        params[kW3 + t] = on ? (t == 0 ? slope(0) : slope(t) - slope(t - 1)) : 0.0f;
    }
    for (int k = t; k < kH * kH; k += blockDim.x) params[kW2 + k] = (k / kH == k % kH) ? 1.0f : 0.0f;
    if (t == 0) params[kB3] = nk > 0 ? ky[0] : 0.0f;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
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
    mlp_init_kernel<<<1, 256, 0, c.stream>>>(c.ly.mlp_x, c.ly.mlp_y, c.ly.mlp_npts, c.ly.mlp_params);
    const int64_t max_pts = std::min<int64_t>(p.sample_size, kMlpTrainPoints);
    const int fgrid = (int)std::max<int64_t>(1, (max_pts + kMlpThreads - 1) / kMlpThreads);
    mlp_features_kernel<<<fgrid, kMlpThreads, 0, c.stream>>>(c.ly.mlp_params, c.ly.mlp_x, c.ly.mlp_npts, c.ly.mlp_part);
    mlp_head_kernel<<<1, kMlpHeadThreads, 0, c.stream>>>(c.ly.mlp_params, c.ly.mlp_part, c.ly.mlp_y, c.ly.mlp_npts,
                                                         kMlpSteps, kMlpLr, c.dbg.mlp_loss ? c.dbg.mlp_loss : nullptr,
                                                         c.dbg.mlp_loss ? c.dbg.mlp_loss + 1 : nullptr);
    cudaError_t e = cudaGetLastError();
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
