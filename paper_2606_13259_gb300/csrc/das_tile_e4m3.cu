// das_tile_e4m3.cu -- tile-kernel instances for 8-bit float storage of IQ data
// (E4M3 and E5M2) with a float32 scale per (transmit, element) (8-bit storage
// is the paper's future work, Sec. 6); forward only, float32 arithmetic.
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

#define DAS_E5M2_CASE(FB) \
    case FB: return launch_tile_best<FB, true, ST_E5M2, MODE_FWD>(A, n_chunks, s);

cudaError_t launch_tile_e5m2(const TileArgs &A, int mode, int iq, int fb, int n_chunks, cudaStream_t s) {
    if (mode != MODE_FWD || !iq) return cudaErrorInvalidValue;
    switch (fb) {
        DAS_E5M2_CASE(1)
        DAS_E5M2_CASE(2)
        DAS_E5M2_CASE(4)
        DAS_E5M2_CASE(8)
        DAS_E5M2_CASE(12)
        DAS_E5M2_CASE(16)
        DAS_E5M2_CASE(20)
        DAS_E5M2_CASE(24)
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace das
