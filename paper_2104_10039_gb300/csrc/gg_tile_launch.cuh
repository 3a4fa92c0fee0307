// gg_tile_launch.cuh - persistent launches of the tile kernels (included by
// the instantiation units).
#pragma once

#include "gg_gather.cuh"
#include "gg_tile.cuh"

namespace gg {

// Persistent grid of `kernel`: as many blocks as fit at once (each warp then
// walks its tiles t, t + W, ...), never more than there are tiles for. The
// occupancy query runs once per kernel (`blocks` is the caller's cache).
static cudaError_t launch_persistent(void (*kernel)(TileArgs), int &blocks, const TileArgs &a, int max_tiles,
                                     int num_sms, cudaStream_t s)
{
    if (blocks == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kThreads, 0) != cudaSuccess || b < 1) b = 1;
        blocks = b;
    }
    int g = blocks * num_sms;
    const int need = (max_tiles + kWarps - 1) / kWarps;
    g = g < need ? g : (need > 0 ? need : 1);
    kernel<<<g, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// The pull gather of an approximate or accurate iteration.
template <int APP>
static cudaError_t launch_gather(const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s)
{
    static int blocks = 0;
    return launch_persistent(k_arcs<APP, K_GATHER>, blocks, a, max_tiles, num_sms, s);
}

// A correction iteration: the stashing gather, then k_correct2 (running-prefix
// influence) or, for PageRank with the share influence, k_share.
template <int APP>
static cudaError_t launch_correction(const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s)
{
    static int b_stash = 0, b_correct = 0, b_share = 0;
    cudaError_t e = launch_persistent(k_arcs<APP, K_STASH>, b_stash, a, max_tiles, num_sms, s);
    if (e != cudaSuccess) return e;
    if constexpr (APP == GG_APP_PAGERANK) {
        if (a.infl_share) return launch_persistent(k_share<APP>, b_share, a, max_tiles, num_sms, s);
    }
    return launch_persistent(k_correct2<APP>, b_correct, a, max_tiles, num_sms, s);
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
