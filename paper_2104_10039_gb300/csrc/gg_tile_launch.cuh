// gg_tile_launch.cuh - cooperative persistent launch of one tile-kernel
// instantiation (included by the instantiation units).
#pragma once

#include "gg_tile.cuh"

namespace gg {

// Co-resident blocks of k_tile<APP, KIND> on this device (cached).
template <int APP, int KIND>
static int resident_blocks(int num_sms)
{
    static int blocks = 0;
    if (blocks == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_tile<APP, KIND>, kThreads, 0) != cudaSuccess || b < 1)
            b = 1;
        blocks = b;
    }
    return blocks * num_sms;
}

// Persistent grid: as many blocks as fit at once (each warp then walks its
// tiles t, t + W, ...), never more than there are tiles for.
template <int APP, int KIND>
static cudaError_t launch_tiles(const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s)
{
    int g = resident_blocks<APP, KIND>(num_sms);
    const int need = (max_tiles + kWarps - 1) / kWarps;
    g = g < need ? g : (need > 0 ? need : 1);
    k_tile<APP, KIND><<<g, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// A correction iteration: K_STASH, then k_correct2 (running-prefix
// influence) or K_CORRECT (the share influence, which needs whole rows).
template <int APP>
static cudaError_t launch_correction(const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s)
{
    cudaError_t e = launch_tiles<APP, K_STASH>(a, max_tiles, num_sms, s);
    if (e != cudaSuccess) return e;
    if (a.infl_share) return launch_tiles<APP, K_CORRECT>(a, max_tiles, num_sms, s);
    static int blocks = 0;
    if (blocks == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_correct2<APP>, kThreads, 0) != cudaSuccess || b < 1)
            b = 1;
        blocks = b;
    }
    int g = blocks * num_sms;
    const int need = (max_tiles + kWarps - 1) / kWarps;
    g = g < need ? g : (need > 0 ? need : 1);
    k_correct2<APP><<<g, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <int APP>
static cudaError_t launch_fixup_app(const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s)
{
    long long blocks = ((long long)max_tiles + kThreads - 1) / kThreads;
    if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
    if (blocks < 1) blocks = 1;
    k_fixup<APP><<<(unsigned)blocks, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gg
