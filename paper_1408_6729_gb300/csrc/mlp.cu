// mlp.cu -- the learned bucket classifier on the GPU: the training set from
// the sorted sample, the spline start, full-batch gradient descent with
// backtracking on every parameter (the forward and backward pass of
// mlp_cta_grad, checked against
// the CPU oracle through bsps_mlp_loss_grad), the evaluation tables of the
// trained network, and the index over the splitters' outputs.
#include <algorithm>

#include "mlp.cuh"

namespace bsps {

constexpr int kMlpThreads = 128;       // one training point per thread per step
constexpr int kMlpMaxPoints = kMlpPointsMax;
// Full-batch gradient descent on all 1153 parameters from the (balanced)
// spline start, with backtracking: each step goes from the best parameters
// so far along their negative gradient; a step that lowers the loss is kept
// and the step size grows, else it is dropped and the step size shrinks.
// The first step size is a tenth of loss / |gradient|^2 (the linear model's
// step to a tenth of the loss).
constexpr int kMlpSteps = 8;
constexpr float kMlpFirst = 0.1f, kMlpGrow = 1.5f, kMlpShrink = 0.25f;
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

// One training step's partial gradients: as mlp_grad_kernel, with the point
// count read from the device (CTAs past it contribute zeros).
__global__ void __launch_bounds__(kMlpThreads) mlp_step_grad_kernel(const float *params, const float *x,
                                                                    const float *y, const int64_t *npts,
                                                                    float *part) {
    __shared__ float w[kParams + 3];
    __shared__ float scratch[kMlpScratchFloats];
    for (int k = threadIdx.x; k < kParams; k += kMlpThreads) w[k] = params[k];
    __syncthreads();
    const int64_t m = *npts;
    const int64_t p0 = (int64_t)blockIdx.x * kMlpThreads;
    float *pp = part + (int64_t)blockIdx.x * (kParams + 1);
    if (p0 >= m) {
        for (int k = threadIdx.x; k <= kParams; k += kMlpThreads) pp[k] = 0.0f;
        return;
    }
    const int np = (int)imin64(kMlpThreads, m - p0);
    const float lp = mlp_cta_grad(w, x, y, p0, np, m, pp, scratch);
    if (threadIdx.x == 0) pp[kParams] = lp;
}

// Descent state: the best parameters, their loss and gradient, the step size.
struct MlpOpt {
    float best[kParams], grad[kParams], start[kParams];
    float best_loss, eta;
};
// the descent state, then (16-byte aligned) the scratch of the evaluation form
static size_t mlp_scratch_offset() { return (sizeof(MlpOpt) + 15) & ~size_t(15); }

// Sums the G partial gradients and losses of the current parameters; keeps
// them as the best if their loss is the lowest so far (the step size grows)
// or drops them (it shrinks); then, unless `last`, sets the parameters to the
// next trial, best - eta * grad(best).  After the last evaluation the best
// parameters are written back.
__global__ void __launch_bounds__(1024) mlp_descent_kernel(float *params, const float *part, int G,
                                                           const int64_t *npts, MlpOpt *opt, int step, int last,
                                                           float *loss_first, float *loss_last) {
    __shared__ float s_loss, s_red[32];
    __shared__ int s_keep;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t m = *npts;
    if (m == 0) return;
    if (t == 0) {
        float l = 0.0f;
        for (int c = 0; c < G; ++c) l += part[(int64_t)c * (kParams + 1) + kParams];
        s_loss = l / (float)m;
        s_keep = step == 0 || s_loss < opt->best_loss;
    }
    __syncthreads();
    const bool keep = s_keep;
    float g2 = 0.0f;
    for (int k = t; k < kParams; k += 1024) {
        if (step == 0) opt->start[k] = params[k];
        if (keep) {
            float g = 0.0f;
            for (int c = 0; c < G; ++c) g += part[(int64_t)c * (kParams + 1) + k];
            opt->best[k] = params[k];
            opt->grad[k] = g;
            g2 = fmaf(g, g, g2);
        }
    }
    // |grad|^2 for the first step size
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) g2 += __shfl_xor_sync(0xffffffffu, g2, o);
    if (lane == 0) s_red[warp] = g2;
    __syncthreads();
    if (t == 0) {
        if (step == 0) {
            float tot = 0.0f;
            for (int w = 0; w < 32; ++w) tot += s_red[w];
            opt->eta = tot > 0.0f ? kMlpFirst * s_loss / tot : 0.0f;
            if (loss_first) *loss_first = s_loss;
        } else {
            opt->eta *= keep ? kMlpGrow : kMlpShrink;
        }
        if (keep) opt->best_loss = s_loss;
        if (last && loss_last) *loss_last = opt->best_loss;
    }
    __syncthreads();
    const float eta = opt->eta;
    for (int k = t; k < kParams; k += 1024)
        params[k] = last ? opt->best[k] : opt->best[k] - eta * opt->grad[k];
}

// The piecewise-linear form of the network `params` (see MlpTables), in
// double, in two kernels.  mlp_pieces_kernel: one warp (CTA) per layer-1
// interval k (between its sorted knots k-1 and k) of each parameter set --
// the trained network and the `fallback` -- lane i taking layer 2's unit i:
// the lane forms the unit's affine pre-activation there and its zero
// crossing; the crossings inside the interval cut it into pieces, and for
// every piece the warp sums the active units' slopes and values at the
// piece's anchor.  (One warp per interval on separate SMs: the double
// arithmetic of all intervals on one SM took 0.12 ms.)  mlp_tables_kernel
// then writes the pieces of all intervals in order; a network of more than
// kMlpPieces pieces is replaced by the fallback (the spline start, at most 33
// pieces), when given.
struct MlpPieceSet {
    double knots[kH];
    int nk;
    int n[kH + 1];
    float x[kH + 1][kH + 1], y[kH + 1][kH + 1], s[kH + 1][kH + 1];
};
struct MlpPieceScratch {
    MlpPieceSet set[2];  // the trained parameters, the fallback
};

__global__ void __launch_bounds__(32) mlp_pieces_kernel(const float *params_in, const float *fallback,
                                                        MlpPieceScratch *scr) {
    const int which = blockIdx.x / (kH + 1), k = blockIdx.x % (kH + 1), lane = threadIdx.x;
    const float *params = which == 0 ? params_in : fallback;
    if (!params) return;
    MlpPieceSet &S = scr->set[which];
    __shared__ double knots[kH];
    __shared__ double cutd[kH + 1];
    __shared__ int nk;
    const double INF = __longlong_as_double(0x7ff0000000000000ll);
    if (lane == 0) {
        int c = 0;
        for (int j = 0; j < kH; ++j) {
            const double w = params[kW1 + j];
            if (w != 0.0) {  // insertion into the sorted list
                const double v = -(double)params[kB1 + j] / w;
                int q = c++;
                while (q > 0 && knots[q - 1] > v) { knots[q] = knots[q - 1]; --q; }
                knots[q] = v;
            }
        }
        nk = c;
        if (k == 0) {
            S.nk = c;
            for (int j = 0; j < c; ++j) S.knots[j] = knots[j];
        }
    }
    __syncwarp();
    const int c = nk;
    if (k > c) {
        if (lane == 0) S.n[k] = 0;
        return;
    }
    const double w3 = params[kW3 + lane];
    const double lo = k == 0 ? -INF : knots[k - 1], hi = k == c ? INF : knots[k];
    // a point inside the interval decides which layer-1 units are on
    double xm = 0.0;
    if (c > 0) xm = k == 0 ? knots[0] - 1.0 : (k == c ? knots[c - 1] + 1.0 : 0.5 * (lo + hi));
    double A = params[kB2 + lane], B = 0.0;  // unit `lane` of layer 2: A + B x here
    for (int j = 0; j < kH; ++j) {
        const double w1 = params[kW1 + j], b1 = params[kB1 + j];
        if (w1 * xm + b1 > 0.0) {
            const double w2 = params[kW2 + lane * kH + j];
            A += w2 * b1;
            B += w2 * w1;
        }
    }
    // its zero crossing, when inside the interval, ranked among the others
    const double z = B != 0.0 ? -A / B : 0.0;
    const bool in = B != 0.0 && z > lo && z < hi;
    const uint32_t valid = __ballot_sync(0xffffffffu, in);
    int rank = 0;
    for (int q = 0; q < 32; ++q) {
        const double zq = __shfl_sync(0xffffffffu, z, q);
        rank += ((valid >> q) & 1u) && (zq < z || (zq == z && q < lane));
    }
    if (in) cutd[rank] = z;
    __syncwarp();
    const int m = __popc(valid);
    // piece r of the interval: [left_r, right_r)
    for (int r = 0; r <= m; ++r) {
        const double left = r == 0 ? lo : cutd[r - 1], right = r == m ? hi : cutd[r];
        double mid, anchor;
        if (left == -INF && right == INF) { mid = 0.0; anchor = 0.0; }
        else if (left == -INF) { mid = right - 1.0; anchor = right; }
        else if (right == INF) { mid = left + 1.0; anchor = left; }
        else { mid = 0.5 * (left + right); anchor = left; }
        const bool on = A + B * mid > 0.0;
        double y = on ? w3 * (A + B * anchor) : 0.0, sl = on ? w3 * B : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            y += __shfl_xor_sync(0xffffffffu, y, o);
            sl += __shfl_xor_sync(0xffffffffu, sl, o);
        }
        if (lane == 0) {
            y += params[kB3];
            // a finite piece over which the network falls by less than
            // 2^-30 (far below the output's float resolution and its
            // index cells) is taken as flat
            if (sl < 0.0 && left != -INF && right != INF && -sl * (right - left) < 9.313225746154785e-10) sl = 0.0;
            S.x[k][r] = (float)anchor;
            S.y[k][r] = (float)y;
            S.s[k][r] = (float)sl;
        }
    }
    if (lane == 0) S.n[k] = m + 1;
}

constexpr int kTablesThreads = 1024;
__global__ void __launch_bounds__(kTablesThreads) mlp_tables_kernel(const MlpPieceScratch *scr, int has_fallback,
                                                                    const MlpNorm *norm, MlpTables *T) {
    __shared__ float s_x[kMlpPiecesAll], s_y[kMlpPiecesAll], s_s[kMlpPiecesAll];
    __shared__ int s_n[kH + 1], s_off[kH + 2];
    __shared__ double knots[kH];
    __shared__ int use;
    const int t = threadIdx.x;
    if (t == 0) {  // the trained network, unless it has too many pieces and a fallback exists
        int o = 0;
        const MlpPieceSet &S0 = scr->set[0];
        for (int k = 0; k <= S0.nk; ++k) o += S0.n[k];
        use = (o > kMlpPieces && has_fallback) ? 1 : 0;
    }
    __syncthreads();
    const MlpPieceSet &S = scr->set[use];
    const int c = S.nk;
    for (int i = t; i < (kH + 1) * (kH + 1); i += kTablesThreads) {
        const int k = i / (kH + 1), r = i % (kH + 1);
        if (k <= c && r < S.n[k]) {
            s_x[i] = S.x[k][r];
            s_y[i] = S.y[k][r];
            s_s[i] = S.s[k][r];
        }
    }
    for (int k = t; k <= c; k += kTablesThreads) s_n[k] = S.n[k];
    for (int j = t; j < c; j += kTablesThreads) knots[j] = S.knots[j];
    __syncthreads();
    if (t == 0) {
        int o = 0;
        for (int k = 0; k <= c; ++k) { s_off[k] = o; o += s_n[k]; }
        s_off[c + 1] = o;
    }
    __syncthreads();
    if (t == 0) {
        const int o = min(s_off[c + 1], kMlpPieces);
        int npad = 1;
        while (npad < o) npad <<= 1;  // cut points: o - 1 < npad
        T->npieces = o;
        T->npad = npad;
        if (norm) T->norm = *norm;
        // values at the pieces' anchors, made nondecreasing; monotone if no
        // slope is negative (then the running maximum only absorbs rounding)
        bool mono = true;
        for (int k = 0; k <= c; ++k)
            for (int r = 0; r < s_n[k]; ++r) mono &= s_s[k * (kH + 1) + r] >= 0.0f;
        if (mono) {
            float run = -__int_as_float(0x7f800000);
            for (int k = 0; k <= c; ++k)
                for (int r = 0; r < s_n[k]; ++r) {
                    const int q = k * (kH + 1) + r;
                    run = fmaxf(run, s_y[q]);
                    s_y[q] = run;
                }
        }
        T->monotone = mono ? 1 : 0;
    }
    __syncthreads();
    for (int k = t; k <= c; k += kTablesThreads) {
        const int o = s_off[k];
        for (int r = 0; r < s_n[k] && o + r < kMlpPieces; ++r) {
            const int q = k * (kH + 1) + r;
            // the value at the piece's right end: the next piece's anchor value
            float yhi = __int_as_float(0x7f800000);
            if (r + 1 < s_n[k]) yhi = s_y[q + 1];
            else if (k < c) yhi = s_y[(k + 1) * (kH + 1)];
            T->piece[o + r] = make_float4(s_x[q], s_y[q], s_s[q], yhi);
            // left end of every piece but the first: the interval's knot or a cut
            if (o + r > 0) T->cut[o + r - 1] = r == 0 ? (float)knots[k - 1] : s_x[q];
        }
    }
    __syncthreads();
    const int np = min(s_off[c + 1], kMlpPieces);
    for (int q = np - 1 + t; q < kMlpCutsPad; q += kTablesThreads) T->cut[q] = __int_as_float(0x7f800000);
}

// both kernels of the evaluation form
static cudaError_t launch_tables(const float *params, const float *fallback, const MlpNorm *norm, MlpTables *T,
                                 MlpPieceScratch *scr, cudaStream_t st) {
    mlp_pieces_kernel<<<2 * (kH + 1), 32, 0, st>>>(params, fallback, scr);
    mlp_tables_kernel<<<1, kTablesThreads, 0, st>>>(scr, fallback != nullptr, norm, T);
    return cudaGetLastError();
}

// The network's output for every splitter (S_{j+1} at index j).
template <int DT>
__global__ void mlp_ysplit_kernel(const MlpTables *T, const typename KeyTraits<DT>::T *vphi, int64_t nsplit,
                                  float *ys) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nsplit) ys[j] = mlp_eval(*T, mlp_input<DT>(KeyTraits<DT>::inv(vphi[j]), T->norm));
}

// The index over the network's output: ylut[c] = number of splitters whose
// output cell (after a running maximum over the splitters, so that the
// counts grow with c) is below c, for c = 0 .. kYCells.
__global__ void __launch_bounds__(1024) mlp_ylut_kernel(float *ys, int64_t nsplit, uint16_t *ylut) {
    __shared__ float tmp[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // running maximum, in place: 1024 threads over consecutive slices
    const int64_t per = (nsplit + 1023) / 1024;
    const int64_t j0 = (int64_t)t * per, j1 = imin64(nsplit, j0 + per);
    float mx = -__int_as_float(0x7f800000);
    for (int64_t j = j0; j < j1; ++j) mx = fmaxf(mx, ys[j]);
    float run = mx;  // inclusive max scan over threads
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float v = __shfl_up_sync(0xffffffffu, run, o);
        if (lane >= o) run = fmaxf(run, v);
    }
    if (lane == 31) tmp[warp] = run;
    __syncthreads();
    if (warp == 0) {
        float v = tmp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v = fmaxf(v, u);
        }
        tmp[lane] = v;
    }
    __syncthreads();
    float pre = warp > 0 ? tmp[warp - 1] : -__int_as_float(0x7f800000);
    const float excl = __shfl_up_sync(0xffffffffu, run, 1);
    if (lane > 0) pre = fmaxf(pre, excl);
    for (int64_t j = j0; j < j1; ++j) {
        pre = fmaxf(pre, ys[j]);
        ys[j] = pre;
    }
    __syncthreads();
    for (int c = t; c <= kYCells; c += 1024) {
        int64_t lo = 0, hi = nsplit;  // splitters with output cell below c
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int)ycell_of(ys[mid]) < c) lo = mid + 1;
            else hi = mid;
        }
        ylut[c] = (uint16_t)lo;
    }
}

// The network's output for m inputs (the evaluation the classifier uses).
__global__ void mlp_predict_kernel(const MlpTables *T, const float *x, int64_t m, float *y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) y[i] = mlp_eval(*T, x[i]);
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
// (W2 diagonal, b2 = 0; relu is the identity on relu outputs), and the output
// weights are the slope changes at the knots, each unit rescaled so that its
// three weights are equal in size.  Training then refines it.
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
    // unit j, rescaled by a = |w3_j|^(1/3) (relu(a z) = a relu(z)): the same
    // function with its weight carried equally by w1_j, W2_jj and w3_j
    if (t < kH) {
        const bool on = t < segs;
        const float w3 = on ? (t == 0 ? slope(0) : slope(t) - slope(t - 1)) : 0.0f;
        const float a = w3 != 0.0f ? cbrtf(fabsf(w3)) : 1.0f;
        params[kW1 + t] = on ? a : 0.0f;
        params[kB1 + t] = on ? -kx[t] * a : -1.0f;  // unused units stay at zero
        params[kB2 + t] = 0.0f;
        params[kW3 + t] = w3 / (a * a);
        params[kW2 + t * kH + t] = a;
    }
    for (int k = t; k < kH * kH; k += blockDim.x)
        if (k / kH != k % kH) params[kW2 + k] = 0.0f;
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
    // full-batch gradient descent on every parameter: the partial gradients
    // of the current parameters, then the step (kMlpSteps trials after the
    // start's evaluation)
    const int64_t max_pts = std::min<int64_t>(p.sample_size, kMlpTrainPoints);
    const int G = (int)std::max<int64_t>(1, (max_pts + kMlpThreads - 1) / kMlpThreads);
    MlpOpt *opt = reinterpret_cast<MlpOpt *>(c.ly.mlp_opt);
    for (int step = 0; step <= kMlpSteps; ++step) {
        mlp_step_grad_kernel<<<G, kMlpThreads, 0, c.stream>>>(c.ly.mlp_params, c.ly.mlp_x, c.ly.mlp_y,
                                                              c.ly.mlp_npts, c.ly.mlp_part);
        mlp_descent_kernel<<<1, 1024, 0, c.stream>>>(c.ly.mlp_params, c.ly.mlp_part, G, c.ly.mlp_npts, opt, step,
                                                  step == kMlpSteps, c.dbg.mlp_loss ? c.dbg.mlp_loss : nullptr,
                                                  c.dbg.mlp_loss ? c.dbg.mlp_loss + 1 : nullptr);
    }
    // the trained network in its evaluation form, and the index over the
    // splitters' outputs
    cudaError_t e0 = launch_tables(c.ly.mlp_params, opt->start, c.ly.mlp_norm, c.ly.mlp_tables,
                                   reinterpret_cast<MlpPieceScratch *>(reinterpret_cast<unsigned char *>(c.ly.mlp_opt) +
                                                                       mlp_scratch_offset()),
                                   c.stream);
    if (e0 != cudaSuccess) return e0;
    const int64_t nsplit = p.P - 1;
    if (nsplit > 0)
        mlp_ysplit_kernel<DT><<<(unsigned)((nsplit + 255) / 256), 256, 0, c.stream>>>(
            c.ly.mlp_tables, (const K *)c.ly.vphi, nsplit, c.ly.mlp_ysplit);
    mlp_ylut_kernel<<<1, 1024, 0, c.stream>>>(c.ly.mlp_ysplit, nsplit, c.ly.ylut);
    cudaError_t e = cudaGetLastError();
    if (c.dbg.mlp_params)
        e = cudaMemcpyAsync(c.dbg.mlp_params, c.ly.mlp_params, sizeof(float) * kParams, cudaMemcpyDeviceToDevice,
                            c.stream);
    return e != cudaSuccess ? e : cudaGetLastError();
}

int mlp_train_kernels() { return 2 + 2 * (kMlpSteps + 1) + 4; }
size_t mlp_opt_bytes() { return mlp_scratch_offset() + sizeof(MlpPieceScratch); }

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
    *bytes = std::max((size_t)std::max<int64_t>(G, 1) * (kParams + 1) * sizeof(float),
                      ((sizeof(MlpTables) + 15) & ~size_t(15)) + sizeof(MlpPieceScratch)) + 256;
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

extern "C" int bsps_mlp_predict(const float *d_params, const float *d_x, int64_t m, float *d_y, void *d_ws,
                                size_t ws_bytes, void *stream) {
    if (m < 0 || !d_params || (m > 0 && (!d_x || !d_y))) return BSPS_ERR_INVALID_ARG;
    const size_t toff = (sizeof(MlpTables) + 15) & ~size_t(15);
    if (!d_ws || ws_bytes < toff + sizeof(MlpPieceScratch) || ((uintptr_t)d_ws & 15) != 0)
        return BSPS_ERR_WORKSPACE_TOO_SMALL;
    cudaStream_t s = (cudaStream_t)stream;
    MlpTables *T = (MlpTables *)d_ws;
    if (launch_tables(d_params, nullptr, nullptr, T,
                      reinterpret_cast<MlpPieceScratch *>(reinterpret_cast<unsigned char *>(d_ws) + toff),
                      s) != cudaSuccess)
        return BSPS_ERR_CUDA;
    if (m > 0) mlp_predict_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(T, d_x, m, d_y);
    return cudaGetLastError() == cudaSuccess ? BSPS_OK : BSPS_ERR_CUDA;
}
