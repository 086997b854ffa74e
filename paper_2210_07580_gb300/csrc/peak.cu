// Throughput ceiling of the exact squared-distance test (no counterpart in
// the paper), for reporting the ALU utilisation of the distance loops.
//
// The kernel runs the instruction mix of the merge's 32 x 32 warp tiles from
// registers only: a point broadcast by shuffle, d int32 differences, d
// 32 x 32 -> 64-bit squares summed in 64 bits, one compare against eps2.  No
// memory access limits it, so distances per second here bound what any of
// the library's distance loops (which also load their points) can reach.
#include "gdbscan.h"
#include "gd_internal.cuh"

namespace gd {

template <int D>
__global__ void __launch_bounds__(256) dist_peak_kernel(int iters, long long eps2, unsigned* sink) {
    const int lane = lane_id();
    int P[D], Q[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        P[j] = (int)((blockIdx.x * 7u + threadIdx.x * 13u + j * 101u) & 0xffffu);
        Q[j] = (int)((lane * 17u + j * 5u) & 0xffffu);
    }
    unsigned hits = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll 8
        for (int u = 0; u < 32; ++u) {
            int pt[D];
#pragma unroll
            for (int j = 0; j < D; ++j) pt[j] = __shfl_sync(kFull, P[j], u);
            hits += sqdist<D>(pt, Q) <= eps2 ? 1u : 0u;
        }
        // the next round's points differ, so nothing is loop-invariant
#pragma unroll
        for (int j = 0; j < D; ++j) P[j] += 1 + j;
    }
    if (hits == 0xffffffffu) *sink = hits;  // keeps the work observable
}

}  // namespace gd

using namespace gd;

extern "C" gd_status gd_distance_peak(int device, int d, double* per_s) {
    if (d < 1 || d > kMaxD || !per_s) return GD_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return GD_ECUDA;
    constexpr int kBlocks = 152 * 8, kThreads = 256, kIters = 512;
    unsigned* sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    gd_status st = GD_OK;
    if (cudaMalloc((void**)&sink, sizeof(unsigned)) != cudaSuccess) return GD_ENOMEM;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) st = GD_ECUDA;
    auto launch = [&]() {
        switch (d) {
#define GD_PK(DD) \
    case DD: dist_peak_kernel<DD><<<kBlocks, kThreads>>>(kIters, 1000000, sink); break;
            GD_PK(1) GD_PK(2) GD_PK(3) GD_PK(4) GD_PK(5) GD_PK(6) GD_PK(7) GD_PK(8)
#undef GD_PK
        }
    };
    float best = 0.f;
    for (int rep = 0; st == GD_OK && rep < 4; ++rep) {
        cudaEventRecord(a);
        launch();
        cudaEventRecord(b);
        if (cudaEventSynchronize(b) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            st = GD_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;  // the first run warms up
    }
    if (st == GD_OK) *per_s = (double)kBlocks * kThreads * kIters * 32.0 / (best / 1e3);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(sink);
    return st;
}
