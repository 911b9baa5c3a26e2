// Runtime grid size -> compile-time template argument.
#pragma once

#include <type_traits>

#include <cuda_runtime.h>

namespace scint {

template <typename F>
cudaError_t dispatch_n(int n, F&& f) {
    switch (n) {
        case 16: return f(std::integral_constant<int, 16>{});
        case 32: return f(std::integral_constant<int, 32>{});
        case 64: return f(std::integral_constant<int, 64>{});
        case 128: return f(std::integral_constant<int, 128>{});
        case 256: return f(std::integral_constant<int, 256>{});
        case 512: return f(std::integral_constant<int, 512>{});
        case 1024: return f(std::integral_constant<int, 1024>{});
        case 2048: return f(std::integral_constant<int, 2048>{});
        case 4096: return f(std::integral_constant<int, 4096>{});
        case 8192: return f(std::integral_constant<int, 8192>{});
        case 16384: return f(std::integral_constant<int, 16384>{});
        default: return cudaErrorInvalidValue;
    }
}

// Opt a kernel into more than 48 KB of dynamic shared memory, once per process.
template <typename K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace scint
