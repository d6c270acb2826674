// das_tile_f32.cu -- tile-kernel instances for float32 storage (forward,
// sound-speed derivative, term count).
#include "das_tile_tma.cuh"

namespace das {

#define DAS_F32_CASE(FB)                                                                              \
    case FB:                                                                                          \
        if (mode == MODE_FWD)                                                                         \
            return iq ? launch_tile_best<FB, true, ST_F32, MODE_FWD>(A, n_chunks, s)                     \
                      : launch_tile_best<FB, false, ST_F32, MODE_FWD>(A, n_chunks, s);                   \
        return iq ? launch_tile_best<FB, true, ST_F32, MODE_DC>(A, n_chunks, s)                          \
                  : launch_tile_best<FB, false, ST_F32, MODE_DC>(A, n_chunks, s);

cudaError_t launch_tile_f32(const TileArgs &A, int mode, int iq, int fb, int n_chunks, cudaStream_t s) {
    if (mode == MODE_COUNT) return launch_tile_t<1, false, ST_F32, MODE_COUNT>(A, 1, s);
    switch (fb) {
        DAS_F32_CASE(1)
        DAS_F32_CASE(2)
        DAS_F32_CASE(4)
        DAS_F32_CASE(8)
        DAS_F32_CASE(10)
        DAS_F32_CASE(12)
        DAS_F32_CASE(16)
        DAS_F32_CASE(20)
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace das
