// das_dispatch.cu -- selects the tile-kernel instance for (mode, data, storage,
// frames per thread).
#include "das_internal.cuh"

namespace das {

cudaError_t launch_tile_f32(const TileArgs &A, int mode, int iq, int fb, int n_chunks, cudaStream_t s);
cudaError_t launch_tile_f16(const TileArgs &A, int mode, int iq, int fb, int n_chunks, cudaStream_t s);
cudaError_t launch_tile_bf16(const TileArgs &A, int mode, int iq, int fb, int n_chunks, cudaStream_t s);
cudaError_t launch_tile_e4m3(const TileArgs &A, int mode, int iq, int fb, int n_chunks, cudaStream_t s);
cudaError_t launch_tile_e5m2(const TileArgs &A, int mode, int iq, int fb, int n_chunks, cudaStream_t s);

bool tile_fb_supported(int mode, int iq, int store, int fb) {
    (void)iq;
    if (mode == MODE_COUNT) return fb == 1;
    if (store == ST_F32) return fb == 1 || fb == 2 || fb == 4 || fb == 8 || fb == 10 || fb == 12 || fb == 16 || fb == 20;
    if (mode != MODE_FWD) return false;
    if ((store == ST_E4M3 || store == ST_E5M2) && !iq) return false;
    return fb == 1 || fb == 2 || fb == 4 || fb == 8 || fb == 12 || fb == 16 || fb == 20 || fb == 24;
}

bool tile_col_supported(int iq, int store, int fb) {
    // bytes per sample; the same rule as ColShape in das_tile.cuh
    const int sz = (iq ? 2 : 1) * (store == ST_F32 ? 4 : (store == ST_E4M3 || store == ST_E5M2) ? 1 : 2);
    const int fg = (fb % 4 == 0 && (4 * sz) % 16 == 0) ? 4 : fb;
    return fb >= 1 && (fb * sz) % 16 == 0 && (fg * sz) % 16 == 0;
}

cudaError_t launch_tile(const TileArgs &A, int mode, int iq, int store, int fb, int n_chunks, cudaStream_t s) {
    if (!tile_fb_supported(mode, iq, store, fb)) return cudaErrorInvalidValue;
    if (mode == MODE_COUNT || store == ST_F32) return launch_tile_f32(A, mode, iq, fb, n_chunks, s);
    if (store == ST_F16) return launch_tile_f16(A, mode, iq, fb, n_chunks, s);
    if (store == ST_E4M3) return launch_tile_e4m3(A, mode, iq, fb, n_chunks, s);
    if (store == ST_E5M2) return launch_tile_e5m2(A, mode, iq, fb, n_chunks, s);
    return launch_tile_bf16(A, mode, iq, fb, n_chunks, s);
}

}  // namespace das
