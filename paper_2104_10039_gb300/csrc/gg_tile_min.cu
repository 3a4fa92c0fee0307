// gg_tile_min.cu - SSSP, BFS and CC instantiations of the tile engine (pull
// gather and correction on a min accumulator).
#include "gg_tile_launch.cuh"

namespace gg {

cudaError_t launch_tile_min(int app, int kind, const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s)
{
    switch (app * 2 + (kind == K_CORRECT ? 1 : 0)) {
    case GG_APP_SSSP * 2: return launch_gather<GG_APP_SSSP>(a, max_tiles, num_sms, s);
    case GG_APP_SSSP * 2 + 1: return launch_correction<GG_APP_SSSP>(a, max_tiles, num_sms, s);
    case GG_APP_BFS * 2: return launch_gather<GG_APP_BFS>(a, max_tiles, num_sms, s);
    case GG_APP_BFS * 2 + 1: return launch_correction<GG_APP_BFS>(a, max_tiles, num_sms, s);
    case GG_APP_CC * 2: return launch_gather<GG_APP_CC>(a, max_tiles, num_sms, s);
    case GG_APP_CC * 2 + 1: return launch_correction<GG_APP_CC>(a, max_tiles, num_sms, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fixup_pr(const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s);

cudaError_t launch_fixup(int app, const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s)
{
    switch (app) {
    case GG_APP_PAGERANK: return launch_fixup_pr(a, max_tiles, num_sms, s);
    case GG_APP_SSSP: return launch_fixup_app<GG_APP_SSSP>(a, max_tiles, num_sms, s);
    case GG_APP_BFS: return launch_fixup_app<GG_APP_BFS>(a, max_tiles, num_sms, s);
    case GG_APP_CC: return launch_fixup_app<GG_APP_CC>(a, max_tiles, num_sms, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gg
