// classify.cuh -- bucket of a key: #{i : S_i <= key} (Fig. 2 step 9) with the
// tie-break of Sec. 5.1.1 (equal keys compare by input position).
#pragma once

#include "kernels.cuh"

namespace bsps {

// The splitters are sorted by (phi, tag).  A radix index over the top bits of
// phi - base resolves the first levels of the search: all splitters whose phi
// lies below cell c are counted by lut[c], all splitters above cell c are
// excluded by lut[c+1], and a binary search decides among the splitters that
// share the key's cell.  The result is exactly the splitter-tree descent.
template <typename K>
__device__ __forceinline__ uint32_t classify_key(K phi, uint32_t tag, const LutParams<K> &lp,
                                                 const uint16_t *lut, const K *sphi,
                                                 const uint32_t *stag) {
    if (phi < lp.base) return 0;
    const K d = phi - lp.base;
    if (d > lp.span) return lp.nsplit;
    const uint32_t c = (uint32_t)(d >> lp.shift);
    uint32_t lo = lut[c], hi = lut[c + 1];
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const K sp = sphi[mid];
        bool le = sp < phi;
        if (sp == phi) le = stag[mid] <= tag;  // tags are read on ties only
        lo = le ? mid + 1 : lo;
        hi = le ? hi : mid;
    }
    return lo;
}

} // namespace bsps
