// cluster.cuh -- reductions over a thread-block cluster (distributed shared memory).
#pragma once

#include <cooperative_groups.h>

namespace sdd {

namespace cg = cooperative_groups;

constexpr int SOLVE_THREADS = 512;
constexpr int SOLVE_WARPS = SOLVE_THREADS / 32;

// Sum of two values over the whole cluster: warps by shuffles, the block's
// warps by thread 0 in order, the cluster's blocks by warp 0 (lane q reads
// block q through distributed shared memory, then a fixed butterfly); every
// thread of every block gets the same bits. Two slot sets alternate between calls: a block
// rewrites a slot set only after the next call's cluster barrier, which every
// block reaches only after it has read the slot set of the call before.
template <typename T>
struct ClusterSlots {
    T warp_part[2][SOLVE_WARPS];
    T block_part[2];
    T total[2];
};

template <typename T>
__device__ __forceinline__ void cluster_sum2(cg::cluster_group& cl, ClusterSlots<T> (&sh)[2], int& seq, T& v0,
                                             T& v1)
{
    ClusterSlots<T>& S = sh[seq & 1];
    ++seq;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, off);
        v1 += __shfl_xor_sync(0xffffffffu, v1, off);
    }
    if (lane == 0) {
        S.warp_part[0][warp] = v0;
        S.warp_part[1][warp] = v1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T t0 = 0, t1 = 0;
        for (int q = 0; q < SOLVE_WARPS; ++q) {
            t0 += S.warp_part[0][q];
            t1 += S.warp_part[1][q];
        }
        S.block_part[0] = t0;
        S.block_part[1] = t1;
    }
    cl.sync();
    if (warp == 0) {
        // lane q reads block q's partials (one round trip), then a fixed butterfly
        const int C = (int)cl.num_blocks();
        T t0 = 0, t1 = 0;
        if (lane < C) {
            const T* rem = cl.map_shared_rank(&S.block_part[0], lane);
            t0 = rem[0];
            t1 = rem[1];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            t0 += __shfl_xor_sync(0xffffffffu, t0, off);
            t1 += __shfl_xor_sync(0xffffffffu, t1, off);
        }
        if (lane == 0) {
            S.total[0] = t0;
            S.total[1] = t1;
        }
    }
    __syncthreads();
    v0 = S.total[0];
    v1 = S.total[1];
}

// The same for four values (one cluster barrier for two pairs of sums).
template <typename T>
struct ClusterSlots4 {
    T warp_part[4][SOLVE_WARPS];
    T block_part[4];
    T total[4];
};

template <typename T>
__device__ __forceinline__ void cluster_sum4(cg::cluster_group& cl, ClusterSlots4<T> (&sh)[2], int& seq, T (&v)[4])
{
    ClusterSlots4<T>& S = sh[seq & 1];
    ++seq;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) S.warp_part[k][warp] = v[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        T t = 0;
        for (int q = 0; q < SOLVE_WARPS; ++q) t += S.warp_part[threadIdx.x][q];
        S.block_part[threadIdx.x] = t;
    }
    cl.sync();
    if (warp == 0) {
        const int C = (int)cl.num_blocks();
        T t[4] = {0, 0, 0, 0};
        if (lane < C) {
            const T* rem = cl.map_shared_rank(&S.block_part[0], lane);
#pragma unroll
            for (int k = 0; k < 4; ++k) t[k] = rem[k];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int k = 0; k < 4; ++k) t[k] += __shfl_xor_sync(0xffffffffu, t[k], off);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) S.total[k] = t[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = S.total[k];
}

}  // namespace sdd
