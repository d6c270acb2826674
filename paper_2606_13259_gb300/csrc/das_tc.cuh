// das_tc.cuh -- arguments and launchers of the tensor-core forward path
// (das_tc.cu).  Not part of the public C-ABI.
#pragma once

#include "das_internal.cuh"

namespace das {

// Sub-items of one tensor-memory accumulation chain unless the tuning sets it
// (applied to plans of at least TC_CHAIN_MIN_TX transmits, whose tiles sum
// the most sub-items; one chain per tile otherwise).
constexpr int TC_CHAIN_DEFAULT = 1024;
constexpr int TC_CHAIN_MIN_TX = 4;

// Arguments of the tensor-core forward kernel (das_tc.cu).
struct TcArgs {
    GridDesc g;
    int M, Q, K;
    int B;            // frames in this call
    int bc;           // frames per chunk: MMA columns 0..bc-1 carry real parts, bc..2bc-1 imaginary parts
    int n;            // MMA N: 2 bc rounded up to a multiple of 16 (<= 256)
    int sb;           // window stages in shared memory
    int sa;           // weight stages in tensor memory (a multiple of hand)
    int hand;         // sub-items per hand-off between the roles (1 or 2; divides sa and sb)
    int list_cap;     // sub-items per work list
    int chain;        // sub-items per accumulation chain before D is added into x (0: one chain)
    int ncols;        // tensor-memory columns the CTA allocates
    float a;          // fs / c
    double ad;
    float theta, hr, hi, thr, tile_radius;
    float er, ei;         // e^{-i theta}
    float ahx, ahy, ahz;  // a times the half extents of the tile's voxel-centre box
    float aR;             // a times the tile radius
    float aR2h;           // a R^2 / 2
    const double *elem_pos;
    const float4 *elem_nrm;
    const int *tx_tb;
    const float *tx_t;
    const float *tx_tmin;
    const float *tx_tmax;
    const float *w_tx;
    const float *ratio;   // [Q][M] weight factor sqrt(scale / largest scale)
    const float *smax;    // the largest storage scale
    int *err;             // bit 2: a wait timed out; bit 3: an item needed more windows than a list holds
    unsigned long long wait_ns;  // limit of the pipeline waits (0: 1 s)
    int probe;            // test hook: the first CTA waits on a barrier nothing arrives on
    unsigned long long *items;  // running count of MMA sub-items (128 x n x 32 each)
    float2 *x;            // image [B][N]
};

// Tensor-core path: channel data y[b][qm][k] (complex64) -> operand layout
// z[c][qm][n/8][2][K][8] of 16-bit values (see das_tc.cu), the per-(q, m)
// weight factors, the samples' factors (zinv) and the largest scale.
cudaError_t launch_tc_stage(const void *y, void *z, const float2 *rot, const float *scale, float *zinv,
                            float *ratio, float *smax, int bf16, int B, int bc, int nch, int n, int QM, int K,
                            cudaStream_t s);
cudaError_t launch_tc(const TcArgs &args, int bf16, const void *z, int nch, int ctas_per_sm, cudaStream_t s);
// MMA width and frames per chunk of the tensor-core path for a call of B
// frames, at most max_bc (<= 128) frames per chunk.
void tc_shape(int B, int max_bc, int &bc, int &nch, int &n);
// Frames per chunk: 128 (N up to 256, one CTA per SM), 112 when two CTAs per
// SM are asked for (N <= 224 leaves room for the weight stages), 48 with three
// or four (N <= 96 in 128 tensor-memory columns).
inline int tc_max_frames(int ctas_per_sm) { return ctas_per_sm >= 3 ? 48 : ctas_per_sm == 2 ? 112 : 128; }
cudaError_t launch_scale(const void *y, float *scale, float *inv_scale, int iq, int store, int B, int QM, int K,
                         cudaStream_t s);

}  // namespace das
