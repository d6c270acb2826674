// das_internal.cuh -- device-side definitions shared by the kernels of the
// GB300 delay-and-sum library (sm_103a).  Not part of the public C-ABI.
//
// Delay arithmetic (Sec. 2, Eq. 1; all float work stays far from the absolute
// delay, which float32 cannot hold to the 1e-5 relative accuracy asked of the
// image):
//
//   tau_s(n, m, q) = a * (T_q(p_n) + ||p_n - r_m||),   a = fs / c   [samples]
//
// The grid is cut into tiles of 8 x 4 x 4 voxels with centre p0.  For every
// (tile, element) the kernel evaluates, in float64 once,
//     a * ||p0 - r_m|| = Rb + rf       (Rb integer, 0 <= rf < 1),
// and for every voxel the cancellation-free float32 difference
//     ||p - r|| - ||p0 - r|| = (2 (p0 - r) . D + |D|^2) / (||p - r|| + ||p0 - r||),
// with D = p - p0 (a few tenths of a millimetre).  The transmit term is kept
// the same way, per (tile, transmit) integer base plus a small float32 rest per
// voxel, built in float64 by the prepare kernel.  The delay in samples is then
//     tau_s = (Rb + Tb) + f,    f = rf + t + delta   (|f| of order 10),
// so k = (Rb + Tb) + floor(f) is exact and alpha = f - floor(f) carries the
// float32 rounding of a number of order 10, about 1e-6 sample.
//
// IQ phase: the relayout multiplies sample k by e^{i theta k} (theta = 2 pi
// f_d / fs, from a float64 table), so the kernels only rotate by the
// fractional part: y[k] e^{i theta tau} = z[k] e^{i theta alpha} and
// y[k+1] e^{i theta tau} = z[k+1] e^{-i theta (1 - alpha)}.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace das {

constexpr int TILE_X = 8;
constexpr int TILE_Y = 4;
constexpr int TILE_Z = 4;
constexpr int TILE_N = TILE_X * TILE_Y * TILE_Z;  // 128 voxels, one per thread
constexpr float APERTURE_MARGIN = 1e-6f;

enum Store { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2, ST_E4M3 = 3, ST_E5M2 = 4 };
enum Mode { MODE_FWD = 0, MODE_DC = 1, MODE_COUNT = 2 };

struct GridDesc {
    int nx, ny, nz;
    int tiles_x, tiles_y, tiles_z;
    long long n_voxels;
    double ox, oy, oz;   // origin
    double sx, sy, sz;   // spacing
};

__host__ __device__ inline long long n_tiles(const GridDesc &g) {
    return (long long)g.tiles_x * g.tiles_y * g.tiles_z;
}

// Centre of tile (tx, ty, tz), float64.
__host__ __device__ inline void tile_centre(const GridDesc &g, int tx, int ty, int tz, double &x, double &y,
                                            double &z) {
    x = g.ox + g.sx * (tx * TILE_X + 0.5 * (TILE_X - 1));
    y = g.oy + g.sy * (ty * TILE_Y + 0.5 * (TILE_Y - 1));
    z = g.oz + g.sz * (tz * TILE_Z + 0.5 * (TILE_Z - 1));
}

// Lane l of a tile: warp l / 32 takes z-layer l / 32 (8 x 4 voxels); each
// quarter-warp (8 lanes) covers a 4 x 2 patch, so the lanes that load together
// sit close to each other and mostly need the same sample rows.
__host__ __device__ inline void lane_offset(int l, int &lx, int &ly, int &lz) {
    const int w = l & 7, qd = (l >> 3) & 3;
    lx = (w & 3) | ((qd & 1) << 2);
    ly = (w >> 2) | ((qd >> 1) << 1);
    lz = l >> 5;
}

// Arguments of the tile kernels (forward, sound-speed derivative, term count).
struct TileArgs {
    GridDesc g;
    int M, Q, K;
    int B;         // frames in this call
    int fb;        // frames per CTA chunk (= template FB) = samples per relayouted row
    int umax;      // rows per staged sample window (staged kernels); 0: rows come from global memory
    int w256;      // 1: 256-bit global sample loads where rows allow
    int col;       // 1: z holds each (chunk, q, m) block in column order (LD_COL in das_tile.cuh)
    float win_lo;  // a * tile radius + margin: lower reach of a window below the tile reference (samples)
    double ad;     // fs / c, float64
    float a;       // fs / c, float32
    float theta;   // 2 pi f_d / fs
    float hr, hi;  // e^{i theta / 2}
    float thr;     // (1 + 1e-6) / (2F)^2, or negative for the full aperture
    float tile_radius;
    double inv_c;
    const double *elem_pos;    // [M][3]
    const float4 *elem_nrm;    // [M] (nx, ny, nz, 0)
    const int *tx_tb;          // [tiles][Q] integer transmit base
    const float *tx_t;         // [tiles][Q][128] transmit rest per voxel
    const float *tx_tmin;      // [tiles][Q] smallest transmit rest over the tile's voxels
    const float *w_tx;         // [tiles][Q][128] transmit weight, or null
    const float *scale;        // [Q][M] storage scale, or null
    const void *z;             // channel data [chunk][Q][M][K][fb] (chunk-major)
    int *err;                  // device error flags (bit 0: a staged-copy wait timed out)
    unsigned long long wait_ns;  // staged kernel, test hook: limit of the probe wait (0: 1 s)
    int probe;                 // staged kernel, test hook: the first CTA waits on a barrier nothing arrives on
    void *x;                   // image [B][N] (MODE_FWD)
    const void *gx;            // cotangent [B][N] (MODE_DC)
    double *partial;           // per-CTA partial sums (MODE_DC, MODE_COUNT)
};

// Arguments of the element-major adjoint kernel.
struct AdjArgs {
    GridDesc g;
    int M, Q, K;
    int B;
    int qc;        // transmits per CTA
    int fb;        // frames per CTA
    double ad;
    float a;
    float theta;
    float hr, hi;
    float er, ei;          // e^{-i theta}
    float thr;
    float tile_radius;
    const double *elem_pos;
    const float4 *elem_nrm;
    const int *tx_tb;
    const float *tx_t;
    const float *tx_tmin;  // [tiles][Q] smallest / largest transmit rest over a tile's voxels
    const float *tx_tmax;
    const int2 *tx_span;   // [tiles] transmit row span over all transmits
    int rows;              // sample rows per band: CTA band r owns rows [r * rows, (r + 1) * rows)
    int n_bands;           // bands per (element, transmit chunk)
    int aRi;               // ceil(a x tile radius) + 2: receive offset bound in rows, with margin
    const float *w_tx;
    const float2 *rot;   // [K] e^{i theta k} (IQ), or null
    const void *x;       // image [B][N]
    void *y;             // channel data [B][Q][M][K], public layout
};

// Kernel launchers (defined in the .cu files).
cudaError_t launch_prepare(const GridDesc &g, int Q, const int *kind, const double *vec, const double *off,
                           const double *t0, double ad, int *tx_tb, float *tx_t, float *tx_tmin, float *tx_tmax,
                           int2 *tx_span, cudaStream_t s);
cudaError_t launch_tile(const TileArgs &args, int mode, int iq, int store, int fb, int n_chunks, cudaStream_t s);
cudaError_t launch_adjoint(const AdjArgs &args, int iq, cudaStream_t s);
// Forward kernel with two x-adjacent voxels per thread sharing sample rows
// (das_tile_pair.cuh): float32 IQ rows in column order.
bool pair_supported(int mode, int iq, int store, int fb);
cudaError_t launch_pair(const TileArgs &A, int store, int fb, int n_chunks, cudaStream_t s);
cudaError_t launch_reduce(const double *partial, long long n, double *out, cudaStream_t s);
bool tile_fb_supported(int mode, int iq, int store, int fb);
// Whether rows of fb samples can be read in column order (whole 16-byte
// pieces per row and per register group of the tile kernels).
bool tile_col_supported(int iq, int store, int fb);
// Relayout of public channel data y[b][q][m][k] into the plan scratch
// z[chunk][q][m][K rows of fb samples] (das_prep.cu); col: column order.
cudaError_t launch_relayout(const void *y, void *z, const float2 *rot, const float *inv_scale, int iq, int store,
                            int B, int fb, int nch, int QM, int K, int col, cudaStream_t s);
// Rows of a staged window: every (voxel, element, transmit) of a tile falls in
// [Tb + Rb + floor(rf + tmin - a R), + 4 a R + 3], R the tile radius.
int window_rows(double a_R);

}  // namespace das
