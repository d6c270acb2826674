// das_tile_pair.cu -- instances of the two-voxels-per-thread forward kernel
// (das_tile_pair.cuh): float32 IQ storage in column order.
#include "das_tile_pair.cuh"

namespace das {

bool pair_supported(int mode, int iq, int store, int fb) {
    return mode == MODE_FWD && iq && store == ST_F32 && (fb == 4 || fb == 8 || fb == 12 || fb == 16 || fb == 20);
}

cudaError_t launch_pair(const TileArgs &A, int store, int fb, int n_chunks, cudaStream_t s) {
    if (store != ST_F32 || !A.col) return cudaErrorInvalidValue;
    switch (fb) {
    case 4: return launch_pair_t<4, ST_F32>(A, n_chunks, s);
    case 8: return launch_pair_t<8, ST_F32>(A, n_chunks, s);
    case 12: return launch_pair_t<12, ST_F32>(A, n_chunks, s);
    case 16: return launch_pair_t<16, ST_F32>(A, n_chunks, s);
    case 20: return launch_pair_t<20, ST_F32>(A, n_chunks, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace das
