// das_tile_e4m3.cu -- tile-kernel instances for 8-bit E4M3 storage of IQ data
// with a float32 scale per (transmit, element) (the 8-bit format the paper
// names as future work, Sec. 5); forward only, float32 arithmetic.
#include "das_tile_tma.cuh"

namespace das {

#define DAS_E4M3_CASE(FB) \
    case FB: return launch_tile_best<FB, true, ST_E4M3, MODE_FWD>(A, n_chunks, s);

cudaError_t launch_tile_e4m3(const TileArgs &A, int mode, int iq, int fb, int n_chunks, cudaStream_t s) {
    if (mode != MODE_FWD || !iq) return cudaErrorInvalidValue;
    switch (fb) {
        DAS_E4M3_CASE(1)
        DAS_E4M3_CASE(2)
        DAS_E4M3_CASE(4)
        DAS_E4M3_CASE(8)
        DAS_E4M3_CASE(12)
        DAS_E4M3_CASE(16)
        DAS_E4M3_CASE(20)
        DAS_E4M3_CASE(24)
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace das
