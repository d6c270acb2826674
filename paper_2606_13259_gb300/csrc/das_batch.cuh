// das_batch.cuh -- one persistent launch over several plans (grids of uneven
// size, element and transmit counts) and all their frames.
//
// The work list holds (plan, frame chunk, tile) items, heaviest plans first.
// Every CTA of the persistent grid takes the next item from an atomic counter
// and runs the staged tile body (das_tile_tma.cuh) with that plan's
// arguments, which travel by value in the kernel parameter block (up to
// BATCH_MAX_PLANS plans).  The counter is zeroed before every launch by a
// memset node in the same CUDA graph.  No CTA waits for another, so the
// launch cannot deadlock whatever the number of resident CTAs.
#pragma once

#include "das_tile_tma.cuh"

namespace das {

constexpr int BATCH_MAX_PLANS = 8;

struct BatchParams {
    TileArgs plans[BATCH_MAX_PLANS];
    const int4 *items;  // (plan, chunk, tile, 0)
    int n_items;
    int *counter;
};

// STAGED: the tile body with sample windows staged by bulk copies; else the
// tile body reading rows from global memory.
template <int FB, bool IQ, int ST, bool STAGED>
__global__ void __launch_bounds__(TILE_N, TmaOcc<FB>::v) batch_kernel(const __grid_constant__ BatchParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(P.counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();  // all threads have the item before thread 0 takes the next one
        if (it >= P.n_items) break;
        const int4 w = P.items[it];
        if constexpr (STAGED) {
            if (!tile_tma_body<FB, IQ, ST, MODE_FWD>(P.plans[w.x], w.z, w.y, smem, 0)) break;
        } else {
            tile_body<FB, IQ, ST, MODE_FWD>(P.plans[w.x], w.z, w.y, smem, 0);
        }
    }
}

// Dynamic shared memory of the batch kernel: the largest per-plan need.
inline size_t batch_smem_bytes(const BatchParams &P, int n_plans, int rb, bool staged) {
    size_t m = 0;
    for (int i = 0; i < n_plans; ++i) {
        const size_t b = staged ? tile_tma_smem_bytes(P.plans[i].Q, P.plans[i].w_tx != nullptr, P.plans[i].umax, rb)
                                : tile_smem_bytes(P.plans[i].Q, P.plans[i].w_tx != nullptr);
        m = b > m ? b : m;
    }
    return m;
}

template <int FB, bool IQ, int ST, bool STAGED>
cudaError_t launch_batch_t(const BatchParams &P, int n_plans, int ctas_per_sm, cudaStream_t s) {
    constexpr int RB = FB * SampleSize<IQ, ST>::v;
    const size_t smem = batch_smem_bytes(P, n_plans, RB, STAGED);
    auto kern = batch_kernel<FB, IQ, ST, STAGED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TILE_N, smem)) != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int per_sm = ctas_per_sm > 0 && ctas_per_sm < occ ? ctas_per_sm : occ;
    long long grid = (long long)sms * per_sm;
    if (grid > P.n_items) grid = P.n_items;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, TILE_N, smem, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_batch(const BatchParams &P, int n_plans, int iq, int store, int fb, int ctas_per_sm, int staged,
                         cudaStream_t s);
bool batch_fb_supported(int iq, int store, int fb);

}  // namespace das
