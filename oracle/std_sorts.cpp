// std_sorts.cpp -- the C++ standard library's sorts on plain key arrays, timed
// beside the oracle as a CPU baseline (bench.py).  BENCHMARK INFRASTRUCTURE
// ONLY, like the rest of oracle/: nothing on the product path loads it.
#include <algorithm>
#include <cstdint>

extern "C" {

// sort n keys in place; dtype 0 uint32, 1 int32, 2 float32, 3 float64
// (floats by operator<, which is the key order for inputs without NaN)
int baseline_std_sort(int dtype, void *keys, int64_t n, int stable) {
    if (n < 0) return -1;
    switch (dtype) {
    case 0: {
        auto *k = static_cast<uint32_t *>(keys);
        stable ? std::stable_sort(k, k + n) : std::sort(k, k + n);
        return 0;
    }
    case 1: {
        auto *k = static_cast<int32_t *>(keys);
        stable ? std::stable_sort(k, k + n) : std::sort(k, k + n);
        return 0;
    }
    case 2: {
        auto *k = static_cast<float *>(keys);
        stable ? std::stable_sort(k, k + n) : std::sort(k, k + n);
        return 0;
    }
    case 3: {
        auto *k = static_cast<double *>(keys);
        stable ? std::stable_sort(k, k + n) : std::sort(k, k + n);
        return 0;
    }
    default:
        return -1;
    }
}

}  // extern "C"
