// Host-side helper of the runtime (api.cu, batch.cu): page-locked arrays for the per-strip
// results read back once per strip-solver launch.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace ddnls {

// Page-locked host array (cudaMallocHost): device-to-host copies into it stay asynchronous,
// where a copy into pageable memory would block the host until the stream reaches it.
template <typename T> struct PinnedVec {
    T* p = nullptr;
    size_t n = 0;
    PinnedVec() = default;
    PinnedVec(const PinnedVec&) = delete;
    PinnedVec& operator=(const PinnedVec&) = delete;
    ~PinnedVec() { if (p) cudaFreeHost(p); }
    // false when the allocation fails (the array is then empty)
    bool resize(size_t m) {
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
        if (m == 0) return true;
        if (cudaMallocHost((void**)&p, m * sizeof(T)) != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return false;
        }
        n = m;
        for (size_t i = 0; i < n; ++i) p[i] = T();
        return true;
    }
    bool assign(size_t m, T v) {
        if (!resize(m)) return false;
        for (size_t i = 0; i < n; ++i) p[i] = v;
        return true;
    }
    T* data() { return p; }
    const T* data() const { return p; }
    T& operator[](size_t i) { return p[i]; }
    const T& operator[](size_t i) const { return p[i]; }
    size_t size() const { return n; }
};

}  // namespace ddnls
