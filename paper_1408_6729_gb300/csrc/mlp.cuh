// mlp.cuh -- the learned bucket classifier (not in the paper).
//
// A 1 -> 32 -> 32 -> 1 ReLU network, FP32, estimates the cumulative
// distribution of the keys; it is trained on the sample the method draws
// anyway (Fig. 1 step 4 / Fig. 3 step 4), against the empirical CDF of the
// sorted sample, and is evaluated through its piecewise-linear form.  Its
// output indexes a table of the splitters' own outputs,
// and a search against the true splitters in the indexed range, checked at
// the range's ends, makes every bucket exactly #{i : S_i <= key} (Fig. 2
// step 9) whatever the network predicts.
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

// ---------------------------------------------------------------------------
// Evaluation form of the trained network.  The network is a continuous
// piecewise-linear function of its input x: layer 1's units switch at their
// knots t_j = -b1_j / w1_j, and between two consecutive knots layer 2's
// pre-activations are affine in x, so each of its units switches at most once
// more there.  Cut at all these points, the function is linear on each piece:
//     y(x) = y_p + s_p (x - x_p)     (x_p: the piece's anchor, y_p = y(x_p)),
// with y_p and s_p computed in double from the trained weights.  A key finds
// its piece by a fixed-depth search over the sorted cut points and is
// evaluated by one fused multiply-add: the network's own function, with an
// error set by x's rounding alone (a piece over which the network falls by
// less than 2^-30 is taken as flat).  When every slope is >= 0 the value is
// also clamped to the piece's two end values, stored once (shared by
// neighbouring pieces) and made nondecreasing, so that the evaluated function
// is then exactly nondecreasing in x.
// ---------------------------------------------------------------------------
constexpr int kYCellBits = 14;                 // cells of the index over the network's output
constexpr int kYCells = 1 << kYCellBits;
constexpr int kMlpPiecesAll = (kH + 1) * (kH + 1);  // at most 33 layer-1 intervals x 33 layer-2 pieces
constexpr int kMlpPieces = 256;                // pieces kept (else the spline start, at most 33, is used)
constexpr int kMlpCutsPad = kMlpPieces;        // cut points, padded to a power of two with +inf
struct MlpTables {
    float cut[kMlpCutsPad];    // ascending left ends of pieces 1 .. np-1, then +inf
    float4 piece[kMlpPieces];  // (x_p, y_p, s_p, y_{p+1}) of piece p = [cut[p-1], cut[p])
    int32_t npieces;
    int32_t npad;              // power of two > npieces - 1 (entries searched)
    int32_t monotone;          // every slope >= 0: the evaluation is nondecreasing
    int32_t pad_;
    MlpNorm norm;
};

__device__ __forceinline__ float mlp_eval(const MlpTables &T, float x) {
    // p = number of cut points <= x (a fixed-depth search)
    int p = 0;
    for (int st = T.npad >> 1; st >= 1; st >>= 1) p += T.cut[p + st - 1] <= x ? st : 0;
    const float4 pc = T.piece[p];
    float y = fmaf(pc.z, x - pc.x, pc.y);
    if (T.monotone) {  // clamped to the piece's end values
        y = fminf(y, pc.w);
        if (p > 0) y = fmaxf(y, pc.y);  // piece 0 extends to -inf; its anchor is its right end
    }
    return y;
}

// Cell of the index over the network's output y (an estimate of the key's
// rank fraction): floor(y * kYCells) clamped to [0, kYCells - 1]; NaN -> 0.
__device__ __forceinline__ uint32_t ycell_of(float y) {
    return (uint32_t)fminf(fmaxf(y * (float)kYCells, 0.0f), (float)(kYCells - 1));
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

// Learned classification (Fig. 2 step 9 with a learned first stage): the
// network's output picks a cell of the index ylut, whose entries count the
// splitters whose own output lies below the cell (outputs made nondecreasing
// by a running maximum).  When the network is nondecreasing the key's bucket
// lies between the cell's two counts; a binary search over those splitters
// finds it.  When the evaluation is exactly nondecreasing (every slope of
// the network >= 0) that is the bucket; otherwise a check against the
// splitters just outside the range makes the result exact whatever the
// network predicts: a key outside the range (a misprediction) is found by
// galloping from there.  `mis` is set for a misprediction; `steps` counts
// the splitter comparisons.
template <int DT>
__device__ __forceinline__ uint32_t classify_learned(typename KeyTraits<DT>::T bits, uint32_t tag,
                                                     const MlpTables &T, const uint16_t *ylut, uint32_t nsplit,
                                                     const typename KeyTraits<DT>::T *sphi, const uint32_t *stag,
                                                     uint32_t &steps, bool &mis) {
    using K = typename KeyTraits<DT>::T;
    const K phi = KeyTraits<DT>::phi(bits);
    auto le = [&](uint32_t j) {
        const K sp = sphi[j];
        return sp < phi || (sp == phi && stag[j] <= tag);
    };
    const float x = mlp_input<DT>(bits, T.norm);
    const uint32_t c = ycell_of(mlp_eval(T, x));
    const uint32_t lo0 = ylut[c], hi0 = ylut[c + 1];
    uint32_t lo = lo0, hi = hi0;
    steps = 0;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        ++steps;
        if (le(mid)) lo = mid + 1;
        else hi = mid;
    }
    // A nondecreasing network (and a finite x) puts the bucket inside the
    // cell's range: a splitter of a lower cell has a lower output, hence a
    // lower x, hence a smaller key.  Otherwise the range is checked.
    mis = false;
    if (T.monotone && fabsf(x) <= 3.4028234663852886e38f) return lo;
    bool ok = true;
    if (lo == lo0 && lo > 0) { ++steps; ok = le(lo - 1); }
    if (ok && lo == hi0 && lo < nsplit) { ++steps; ok = !le(lo); }
    mis = !ok;
    if (ok) return lo;
    uint32_t more;
    const uint32_t b = correct_bucket(lo, phi, tag, nsplit, sphi, stag, more);
    steps += more;
    return b;
}

} // namespace bsps
