// Launch and occupancy of the per-iteration pass kernels, instantiated per
// precision by engine_iter_f32.cu and engine_iter_f64.cu.
#pragma once
#include "engine_csr.cuh"
#include "engine_device.cuh"
#include "engine_lean.cuh"
#include "engine_lean3d.cuh"

namespace ld {

// the lean pass exists for FP32 vectors, tiles of 2 or 4 columns, on 2D lattices
template <typename V, int T, int KIND>
constexpr bool has_lean() {
    return std::is_same<V, float>::value && (T == 2 || T == 4) &&
           (KIND == KIND_2D5 || KIND == KIND_2D13_SQ);
}

// the lean 3D pass: FP32 vectors, tiles of 2 or 4 columns, the 7-point kind
template <typename V, int T, int KIND>
constexpr bool has_lean3d() {
    return std::is_same<V, float>::value && (T == 2 || T == 4) && KIND == KIND_3D7;
}

template <int T>
int lean3d_launch(const Solve &s, dim3 grid, int cur, cudaStream_t st) {
    constexpr size_t sm = lean3d_smem_bytes<float, T>();
    if (s.keep_x0)
        k_lean3d<float, T, true><<<grid, L3T, sm, st>>>(s, cur);
    else
        k_lean3d<float, T, false><<<grid, L3T, sm, st>>>(s, cur);
    return (int)cudaGetLastError();
}

template <int T>
int lean3d_occupancy(int *out, bool keepx) {
    constexpr size_t sm = lean3d_smem_bytes<float, T>();
    if (cudaFuncSetAttribute(k_lean3d<float, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_lean3d<float, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
            cudaSuccess)
        return (int)cudaGetLastError();
    if (keepx)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_lean3d<float, T, true>, L3T, sm);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_lean3d<float, T, false>, L3T, sm);
    return (int)cudaGetLastError();
}

template <int T, int X, int KIND>
int lean_launch(const Solve &s, dim3 grid, int cur, cudaStream_t st) {
    if constexpr (KIND == KIND_2D5) {
        if (s.keep_x0) {
            k_lean2d<T, X, KIND, true><<<grid, LEAN_NT, LeanSmem<T, X, KIND, true>::bytes, st>>>(s, cur);
            return (int)cudaGetLastError();
        }
    }
    k_lean2d<T, X, KIND, false><<<grid, LEAN_NT, LeanSmem<T, X, KIND, false>::bytes, st>>>(s, cur);
    return (int)cudaGetLastError();
}

// resident CTAs per SM of the lean pass (sets the shared-memory opt-in of its variants)
template <int T, int X, int KIND>
int lean_occupancy(int *out, bool keepx) {
    constexpr size_t sm0 = LeanSmem<T, X, KIND, false>::bytes;
    if (cudaFuncSetAttribute(k_lean2d<T, X, KIND, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm0) != cudaSuccess)
        return (int)cudaGetLastError();
    if constexpr (KIND == KIND_2D5) {
        constexpr size_t sm1 = LeanSmem<T, X, KIND, true>::bytes;
        if (cudaFuncSetAttribute(k_lean2d<T, X, KIND, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm1) != cudaSuccess)
            return (int)cudaGetLastError();
        if (keepx) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_lean2d<T, X, KIND, true>, LEAN_NT, sm1);
            return (int)cudaGetLastError();
        }
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_lean2d<T, X, KIND, false>, LEAN_NT, sm0);
    return (int)cudaGetLastError();
}

template <typename V, int T, int KIND>
struct IterLauncher {
    static int run(const Solve &s, int cur, cudaStream_t st) {
        const int ts = s.tstride > 0 ? s.tstride : 1;
        const int nt = s.tile0 < s.ntiles ? (s.ntiles - s.tile0 + ts - 1) / ts : 0;
        if (nt == 0) return 0;
        dim3 grid(s.bpt, nt);
        if constexpr (has_lean3d<V, T, KIND>()) {
            if (s.lean == LEAN_3D) return lean3d_launch<T>(s, grid, cur, st);
        }
        if constexpr (has_lean<V, T, KIND>()) {
            if (s.lean == 1) return lean_launch<T, 1, KIND>(s, grid, cur, st);
            if constexpr (T == 2) {
                if (s.lean == 2) return lean_launch<T, 2, KIND>(s, grid, cur, st);
            }
        }
        if constexpr (KIND == KIND_2D5 || KIND == KIND_2D13_SQ) {
            constexpr int G = stream_groups<V, T>();
            constexpr size_t sm = stream_smem_bytes<V, T, G, KIND>(), smb = stream_bulk_smem_bytes<V, T>();
            if (s.bulk) {
                if (s.keep_x0)
                    k_stream2d<V, T, 1, KIND, true, true><<<grid, SW, smb, st>>>(s, cur);
                else
                    k_stream2d<V, T, 1, KIND, false, true><<<grid, SW, smb, st>>>(s, cur);
            } else if (s.keep_x0) {
                k_stream2d<V, T, G, KIND, true, false><<<grid, SW * G, sm, st>>>(s, cur);
            } else {
                k_stream2d<V, T, G, KIND, false, false><<<grid, SW * G, sm, st>>>(s, cur);
            }
        } else if constexpr (KIND == KIND_3D7) {
            if (s.keep_x0)
                k_stream3d<V, T, true><<<grid, P3T, stream3d_smem_bytes<V, T>(), st>>>(s, cur);
            else
                k_stream3d<V, T, false><<<grid, P3T, stream3d_smem_bytes<V, T>(), st>>>(s, cur);
        } else {   // CSR: the streaming step, then the product with the dots and the tail
            k_csr_step<V, T><<<grid, CSR_NT, 0, st>>>(s, cur);
            k_csr_spmv<V, T><<<grid, CSR_NT, 0, st>>>(s, cur);
        }
        return (int)cudaGetLastError();
    }
};

template <typename V, int T, int KIND>
struct OccLauncher {
    // resident CTAs per SM of the iteration kernels (the smaller of the two phases)
    static int run(int *out, bool bulk, int lean, bool keepx) {
        int a = 0, b = 0;
        if constexpr (has_lean3d<V, T, KIND>()) {
            if (lean == LEAN_3D) return lean3d_occupancy<T>(out, keepx);
        }
        if constexpr (has_lean<V, T, KIND>()) {
            if (lean == 1) return lean_occupancy<T, 1, KIND>(out, keepx);
            if constexpr (T == 2) {
                if (lean == 2) return lean_occupancy<T, 2, KIND>(out, keepx);
            }
        }
        if constexpr (KIND == KIND_2D5 || KIND == KIND_2D13_SQ) {
            constexpr int G = stream_groups<V, T>();
            constexpr size_t sm = stream_smem_bytes<V, T, G, KIND>(), smb = stream_bulk_smem_bytes<V, T>();
            if (cudaFuncSetAttribute(k_stream2d<V, T, G, KIND, false, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
                cudaFuncSetAttribute(k_stream2d<V, T, G, KIND, true, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
                cudaFuncSetAttribute(k_stream2d<V, T, 1, KIND, false, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb) != cudaSuccess ||
                cudaFuncSetAttribute(k_stream2d<V, T, 1, KIND, true, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb) != cudaSuccess)
                return (int)cudaGetLastError();
            if (bulk)
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_stream2d<V, T, 1, KIND, true, true>, SW, smb);
            else
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_stream2d<V, T, G, KIND, true, false>, SW * G, sm);
        } else if constexpr (KIND == KIND_3D7) {
            constexpr size_t sm = stream3d_smem_bytes<V, T>();
            if (cudaFuncSetAttribute(k_stream3d<V, T, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
                cudaFuncSetAttribute(k_stream3d<V, T, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
                return (int)cudaGetLastError();
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_stream3d<V, T, true>, P3T, sm);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_csr_spmv<V, T>, CSR_NT, 0);
        }
        (void)b;
        *out = a;
        return (int)cudaGetLastError();
    }
};

template <typename V>
int iteration_launch(const Solve &s, int cur, cudaStream_t st) {
    return dispatch_v<V, IterLauncher>(s.T, s.op.kind, s, cur, st);
}

template <typename V>
int iteration_occupancy(int T, int kind, bool bulk, int lean, bool keepx, int *occ) {
    return dispatch_v<V, OccLauncher>(T, kind, occ, bulk, lean, keepx);
}

}  // namespace ld
