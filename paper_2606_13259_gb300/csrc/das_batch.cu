// das_batch.cu -- instances of the persistent multi-plan kernel.
#include "das_batch.cuh"

namespace das {

bool batch_fb_supported(int iq, int store, int fb) {
    if (iq) {
        if (store == ST_F32) return fb == 2 || fb == 4 || fb == 8 || fb == 12 || fb == 16 || fb == 20;
        return fb == 4 || fb == 8 || fb == 12 || fb == 16 || fb == 20 || fb == 24;
    }
    return store == ST_F32 && (fb == 4 || fb == 8 || fb == 12 || fb == 16 || fb == 20);
}

#define DAS_BATCH_IQ(FB, ST)                                                        \
    case FB:                                                                        \
        return staged ? launch_batch_t<FB, true, ST, true>(P, n_plans, ctas_per_sm, s) \
                      : launch_batch_t<FB, true, ST, false>(P, n_plans, ctas_per_sm, s);
#define DAS_BATCH_RF(FB)                                                               \
    case FB:                                                                           \
        return staged ? launch_batch_t<FB, false, ST_F32, true>(P, n_plans, ctas_per_sm, s) \
                      : launch_batch_t<FB, false, ST_F32, false>(P, n_plans, ctas_per_sm, s);

cudaError_t launch_batch(const BatchParams &P, int n_plans, int iq, int store, int fb, int ctas_per_sm, int staged,
                         cudaStream_t s) {
    if (!batch_fb_supported(iq, store, fb)) return cudaErrorInvalidValue;
    if (iq && store == ST_F32) {
        switch (fb) { DAS_BATCH_IQ(2, ST_F32) DAS_BATCH_IQ(4, ST_F32) DAS_BATCH_IQ(8, ST_F32)
                      DAS_BATCH_IQ(12, ST_F32) DAS_BATCH_IQ(16, ST_F32) DAS_BATCH_IQ(20, ST_F32) }
    } else if (iq && store == ST_F16) {
        switch (fb) { DAS_BATCH_IQ(4, ST_F16) DAS_BATCH_IQ(8, ST_F16) DAS_BATCH_IQ(12, ST_F16)
                      DAS_BATCH_IQ(16, ST_F16) DAS_BATCH_IQ(20, ST_F16) DAS_BATCH_IQ(24, ST_F16) }
    } else if (iq) {
        switch (fb) { DAS_BATCH_IQ(4, ST_BF16) DAS_BATCH_IQ(8, ST_BF16) DAS_BATCH_IQ(12, ST_BF16)
                      DAS_BATCH_IQ(16, ST_BF16) DAS_BATCH_IQ(20, ST_BF16) DAS_BATCH_IQ(24, ST_BF16) }
    } else {
        switch (fb) { DAS_BATCH_RF(4) DAS_BATCH_RF(8) DAS_BATCH_RF(12) DAS_BATCH_RF(16) DAS_BATCH_RF(20) }
    }
    return cudaErrorInvalidValue;
}

}  // namespace das
