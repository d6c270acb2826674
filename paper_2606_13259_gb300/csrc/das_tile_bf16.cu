// das_tile_bf16.cu -- tile-kernel instances for bf16 storage with a float32
// scale per (transmit, element) (Sec. 3.3, mixed-precision storage); forward only.
#include "das_tile_tma.cuh"

namespace das {

#define DAS_BF16_CASE(FB)                                                                            \
    case FB:                                                                                          \
        return iq ? launch_tile_best<FB, true, ST_BF16, MODE_FWD>(A, n_chunks, s)                       \
                  : launch_tile_best<FB, false, ST_BF16, MODE_FWD>(A, n_chunks, s);

cudaError_t launch_tile_bf16(const TileArgs &A, int mode, int iq, int fb, int n_chunks, cudaStream_t s) {
    if (mode != MODE_FWD) return cudaErrorInvalidValue;
    switch (fb) {
        DAS_BF16_CASE(1)
        DAS_BF16_CASE(2)
        DAS_BF16_CASE(4)
        DAS_BF16_CASE(8)
        DAS_BF16_CASE(12)
        DAS_BF16_CASE(16)
        DAS_BF16_CASE(20)
        DAS_BF16_CASE(24)
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace das
