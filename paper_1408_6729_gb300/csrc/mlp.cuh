// mlp.cuh -- the learned bucket classifier (not in the paper).
//
// A 1 -> 32 -> 32 -> 1 ReLU network, FP32, estimates the cumulative
// distribution of the keys; it is trained on the sample the method draws
// anyway (Fig. 1 step 4 / Fig. 3 step 4), against the empirical CDF of the
// sorted sample.  A key's predicted sub-bucket floor(P * y) is then corrected
// by a bounded search against the true splitters, so the bucket is exactly
// #{i : S_i <= key} (Fig. 2 step 9) whatever the network predicts.
//
// Parameter vector (1153 floats): W1[32] b1[32] W2[32][32] (row i = unit i of
// layer 2) b2[32] w3[32] b3.
#pragma once

#include "kernels.cuh"

namespace bsps {

constexpr int kH = 32;
constexpr int kW1 = 0, kB1 = 32, kW2 = 64, kB2 = 64 + 1024, kW3 = kB2 + 32, kB3 = kW3 + 32;
constexpr int kParams = kB3 + 1;  // 1153
constexpr int kMlpPointsMax = 16384;    // training points taken from the sample
constexpr int kMlpGridMax = 128;        // CTAs of the training launch (128 points each)

// x = (value(key) - lo) * scale, value() the key's numeric value
struct MlpNorm {
    double lo;
    float scale;
    float lo_f;
};

template <int DT> __device__ __forceinline__ float mlp_input(typename KeyTraits<DT>::T bits, const MlpNorm &nm) {
    if constexpr (DT == BSPS_U32) return ((float)bits - nm.lo_f) * nm.scale;
    else if constexpr (DT == BSPS_I32) return ((float)(int32_t)bits - nm.lo_f) * nm.scale;
    else if constexpr (DT == BSPS_F32) return (__uint_as_float(bits) - nm.lo_f) * nm.scale;
    else return (float)(__longlong_as_double((long long)bits) - nm.lo) * nm.scale;
}

template <int DT> __host__ __device__ __forceinline__ double key_value(typename KeyTraits<DT>::T bits) {
    if constexpr (DT == BSPS_U32) return (double)bits;
    else if constexpr (DT == BSPS_I32) return (double)(int32_t)bits;
    else if constexpr (DT == BSPS_F32) {
        union { uint32_t u; float f; } c;
        c.u = bits;
        return (double)c.f;
    } else {
        union { uint64_t u; double d; } c;
        c.u = bits;
        return c.d;
    }
}

// Forward pass for one input; weights in shared (or global) memory.
__device__ __forceinline__ float mlp_forward(const float *__restrict__ w, float x) {
    float h1[kH];
#pragma unroll
    for (int j = 0; j < kH; ++j) h1[j] = fmaxf(fmaf(w[kW1 + j], x, w[kB1 + j]), 0.0f);
    float y = w[kB3];
#pragma unroll 4
    for (int i = 0; i < kH; ++i) {
        const float4 *row = reinterpret_cast<const float4 *>(w + kW2 + i * kH);
        float z = w[kB2 + i];
#pragma unroll
        for (int q = 0; q < kH / 4; ++q) {
            const float4 r = row[q];
            z = fmaf(r.x, h1[4 * q], z);
            z = fmaf(r.y, h1[4 * q + 1], z);
            z = fmaf(r.z, h1[4 * q + 2], z);
            z = fmaf(r.w, h1[4 * q + 3], z);
        }
        y = fmaf(w[kW3 + i], fmaxf(z, 0.0f), y);
    }
    return y;
}

// Exact bucket #{j : S_j <= e} from a predicted one: check the guess against
// its two splitters, gallop towards the key, then binary search.  `steps`
// counts splitter comparisons beyond the two of the check.
template <typename K>
__device__ __forceinline__ uint32_t correct_bucket(uint32_t guess, K phi, uint32_t tag, uint32_t nsplit,
                                                   const K *sphi, const uint32_t *stag, uint32_t &steps) {
    auto le = [&](uint32_t j) {  // S_{j+1} <= e, splitter j (0-indexed)
        const K sp = sphi[j];
        return sp < phi || (sp == phi && stag[j] <= tag);
    };
    uint32_t g = guess;
    steps = 0;
    // answer lies in [lo, hi]
    uint32_t lo, hi;
    if (g > 0 && !le(g - 1)) {
        // answer < g: gallop down over j with le(j) false
        hi = g - 1;
        uint32_t step = 1, probe = g - 1;
        for (;;) {
            ++steps;
            if (probe < step) { lo = 0; break; }
            probe -= step;
            if (le(probe)) { lo = probe + 1; break; }
            hi = probe;
            step <<= 1;
        }
    } else if (g < nsplit && le(g)) {
        // answer > g
        lo = g + 1;
        uint32_t step = 1, probe = g;
        for (;;) {
            ++steps;
            probe += step;
            if (probe >= nsplit) { hi = nsplit; break; }
            if (!le(probe)) { hi = probe; break; }
            lo = probe + 1;
            step <<= 1;
        }
    } else {
        return g;
    }
    // smallest j in [lo, hi] with le(j) false (hi = nsplit means none): answer = that j
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        ++steps;
        if (le(mid)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <int DT>
__device__ __forceinline__ uint32_t classify_learned(typename KeyTraits<DT>::T bits, uint32_t tag, const float *w,
                                                     const MlpNorm &nm, uint32_t P, const typename KeyTraits<DT>::T *sphi,
                                                     const uint32_t *stag, uint32_t &steps) {
    const float y = mlp_forward(w, mlp_input<DT>(bits, nm)) * (float)P;
    uint32_t g = 0;
    if (y >= 1.0f) g = y >= (float)(P - 1) ? P - 1 : (uint32_t)y;  // NaN -> 0
    return correct_bucket(g, KeyTraits<DT>::phi(bits), tag, P - 1, sphi, stag, steps);
}

} // namespace bsps
