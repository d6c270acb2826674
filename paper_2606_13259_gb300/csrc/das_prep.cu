// das_prep.cu -- per-plan preparation and channel-data relayout kernels.
//
//  * prepare: transmit delays (Sec. 2, Eq. 1 footnote) per (tile, transmit) as
//    an integer base in samples plus a float32 rest per voxel, built in float64
//    for the plan's current c.  The paper likewise keeps tau^tx precomputed per
//    voxel while receive delays are computed in-kernel (Sec. 3.1).
//  * scale: per (transmit, element) max |sample| for 16-bit storage (Sec. 3.3).
//  * relayout: y[b][q][m][k] -> z[q][m][k][b] with the batch index innermost
//    (Sec. 3.2, batch-inner layout), fused with the IQ pre-rotation by
//    e^{i theta k} and the conversion to the storage type (Sec. 3.3).
//  * reduce: deterministic sum of per-CTA partials.
#include "das_internal.cuh"

namespace das {

// ---------------------------------------------------------------------------
// prepare
// ---------------------------------------------------------------------------

__device__ inline double tx_path(int kind, double vx, double vy, double vz, double off, double t0x, double t0y,
                                 double t0z, double px, double py, double pz) {
    if (kind == 0) {
        double dx = px - vx, dy = py - vy, dz = pz - vz;
        return sqrt(dx * dx + dy * dy + dz * dz) - off;
    }
    if (kind == 1) return vx * (px - t0x) + vy * (py - t0y) + vz * (pz - t0z);
    return 0.0;
}

// One CTA per tile, one thread per voxel lane.  Also records, per (tile,
// transmit), the smallest and largest float32 rest over the tile's voxels:
// together with the tile radius they bound the sample rows any voxel of the
// tile can need; and per tile the row span of the transmit part over all
// transmits, tb + floor(rest) from its smallest to its largest value + 1.
__global__ void __launch_bounds__(TILE_N) prepare_kernel(GridDesc g, int Q, const int *__restrict__ kind,
                                                         const double *__restrict__ vec,
                                                         const double *__restrict__ off, double t0x, double t0y,
                                                         double t0z, double ad, int *__restrict__ tx_tb,
                                                         float *__restrict__ tx_t, float *__restrict__ tx_tmin,
                                                         float *__restrict__ tx_tmax, int2 *__restrict__ tx_span) {
    __shared__ float red[TILE_N / 32], red_max[TILE_N / 32];
    const long long tile = blockIdx.x;
    const int tx = (int)(tile % g.tiles_x);
    const int ty = (int)((tile / g.tiles_x) % g.tiles_y);
    const int tz = (int)(tile / ((long long)g.tiles_x * g.tiles_y));
    int lx, ly, lz;
    lane_offset(threadIdx.x, lx, ly, lz);
    const bool valid = tx * TILE_X + lx < g.nx && ty * TILE_Y + ly < g.ny && tz * TILE_Z + lz < g.nz;
    double cx, cy, cz;
    tile_centre(g, tx, ty, tz, cx, cy, cz);
    const double px = g.ox + g.sx * (tx * TILE_X + lx);
    const double py = g.oy + g.sy * (ty * TILE_Y + ly);
    const double pz = g.oz + g.sz * (tz * TILE_Z + lz);
    int span_lo = 0x7fffffff, span_hi = -0x7fffffff;  // thread 0: transmit row span over all q
    for (int q = 0; q < Q; ++q) {
        const int kd = kind[q];
        const double vx = vec[3 * q], vy = vec[3 * q + 1], vz = vec[3 * q + 2], o = off[q];
        const double base = floor(ad * tx_path(kd, vx, vy, vz, o, t0x, t0y, t0z, cx, cy, cz));
        const float t = (float)(ad * tx_path(kd, vx, vy, vz, o, t0x, t0y, t0z, px, py, pz) - base);
        tx_t[(tile * Q + q) * TILE_N + threadIdx.x] = t;
        if (threadIdx.x == 0) tx_tb[tile * Q + q] = (int)base;
        float mn = valid ? t : 3.0e38f, mx = valid ? t : -3.0e38f;
        for (int d = 16; d > 0; d >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, d));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, d));
        }
        if ((threadIdx.x & 31) == 0) {
            red[threadIdx.x >> 5] = mn;
            red_max[threadIdx.x >> 5] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = red[0], u = red_max[0];
            for (int w = 1; w < TILE_N / 32; ++w) {
                m = fminf(m, red[w]);
                u = fmaxf(u, red_max[w]);
            }
            tx_tmin[tile * Q + q] = m;
            if (tx_tmax) tx_tmax[tile * Q + q] = u;
            if (m <= u) {  // the tile has voxels inside the grid
                span_lo = min(span_lo, (int)base + (int)floorf(m));
                span_hi = max(span_hi, (int)base + (int)floorf(u) + 1);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && tx_span) tx_span[tile] = make_int2(span_lo, span_hi);
}

cudaError_t launch_prepare(const GridDesc &g, int Q, const int *kind, const double *vec, const double *off,
                           const double *t0, double ad, int *tx_tb, float *tx_t, float *tx_tmin, float *tx_tmax,
                           int2 *tx_span, cudaStream_t s) {
    const long long nt = n_tiles(g);
    prepare_kernel<<<(unsigned)nt, TILE_N, 0, s>>>(g, Q, kind, vec, off, t0[0], t0[1], t0[2], ad, tx_tb, tx_t,
                                                   tx_tmin, tx_tmax, tx_span);
    return cudaGetLastError();
}

int window_rows(double a_R) { return (int)ceil(4.0 * a_R) + 4; }

// ---------------------------------------------------------------------------
// storage conversion helpers
// ---------------------------------------------------------------------------

template <int ST> struct StoreT;
template <> struct StoreT<ST_F32> { using c = float2; using r = float; };
template <> struct StoreT<ST_F16> { using c = __half2; using r = __half; };
template <> struct StoreT<ST_BF16> { using c = __nv_bfloat162; using r = __nv_bfloat16; };
template <> struct StoreT<ST_E4M3> { using c = __nv_fp8x2_storage_t; using r = __nv_fp8_storage_t; };
// E5M2 bytes, as types of their own so that the conversion is chosen by type
struct e5m2_t { __nv_fp8_storage_t v; };
struct e5m2x2_t { __nv_fp8x2_storage_t v; };
template <> struct StoreT<ST_E5M2> { using c = e5m2x2_t; using r = e5m2_t; };

__device__ inline void put(float2 *p, float2 v) { *p = v; }
__device__ inline void put(__half2 *p, float2 v) { *p = __floats2half2_rn(v.x, v.y); }
__device__ inline void put(__nv_bfloat162 *p, float2 v) { *p = __floats2bfloat162_rn(v.x, v.y); }
__device__ inline void put(float *p, float v) { *p = v; }
__device__ inline void put(__half *p, float v) { *p = __float2half_rn(v); }
__device__ inline void put(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ inline void put(__nv_fp8_storage_t *p, float v) { *p = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3); }
__device__ inline void put(__nv_fp8x2_storage_t *p, float2 v) {
    *p = __nv_cvt_float2_to_fp8x2(v, __NV_SATFINITE, __NV_E4M3);
}
__device__ inline void put(e5m2_t *p, float v) { p->v = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E5M2); }
__device__ inline void put(e5m2x2_t *p, float2 v) { p->v = __nv_cvt_float2_to_fp8x2(v, __NV_SATFINITE, __NV_E5M2); }

__device__ inline float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// ---------------------------------------------------------------------------
// scale: per (q, m) row set, the largest |component| over frames and samples
// ---------------------------------------------------------------------------

// The scale maps the largest component to `range` (1 for 16-bit storage, the
// largest finite value of the format for 8-bit storage: 448 E4M3, 57344 E5M2).
template <bool IQ>
__global__ void __launch_bounds__(256) scale_kernel(const float *__restrict__ y, float *__restrict__ scale,
                                                    float *__restrict__ inv_scale, int B, int QM, int K,
                                                    float range) {
    const int qm = blockIdx.x;
    const int comp = IQ ? 2 : 1;
    float mx = 0.f;
    for (int b = 0; b < B; ++b) {
        const float *row = y + ((size_t)b * QM + qm) * (size_t)K * comp;
        for (int i = threadIdx.x; i < K * comp; i += blockDim.x) mx = fmaxf(mx, fabsf(row[i]));
    }
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        mx = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (threadIdx.x == 0) {
            const float s = (mx > 0.f && isfinite(mx)) ? mx / range : 1.f;
            scale[qm] = s;
            inv_scale[qm] = 1.f / s;
        }
    }
}

cudaError_t launch_scale(const void *y, float *scale, float *inv_scale, int iq, int store, int B, int QM, int K,
                         cudaStream_t s) {
    const float range = store == ST_E4M3 ? 448.f : store == ST_E5M2 ? 57344.f : 1.f;
    if (iq) scale_kernel<true><<<QM, 256, 0, s>>>((const float *)y, scale, inv_scale, B, QM, K, range);
    else scale_kernel<false><<<QM, 256, 0, s>>>((const float *)y, scale, inv_scale, B, QM, K, range);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// relayout
// ---------------------------------------------------------------------------

// Byte offset of byte `rb` of row k inside a (chunk, q, m) block of K rows of
// RB bytes: row order (k * RB + rb), or column order (16-byte piece rb / 16 of
// every row in one column of K pieces: (rb / 16) * K * 16 + k * 16 + rb % 16).
__device__ __forceinline__ size_t row_byte(int k, int rb, int K, int RB, bool col) {
    return col ? (size_t)(rb >> 4) * ((size_t)K * 16) + (size_t)k * 16 + (rb & 15) : (size_t)k * RB + rb;
}

// Batched: 32 frames x 32 samples per step through shared memory; reads are
// contiguous along k, writes contiguous along the frames of a chunk.  The
// output is chunk-major, z[c][qm][K rows of fb samples] holding frame
// b = c * fb + j, so the rows one CTA of the tile kernels reads lie in one
// block.  For IQ data and an even fb a row is stored pair-planar (re_0, re_1,
// im_0, im_1, re_2, ...), so the kernels can update two frames with one packed
// float32 FMA.  With `col` each block is stored in column order (row_byte).
// Frames B .. Bs-1 (Bs = chunks * fb) are zero.
template <bool IQ, int ST>
__global__ void __launch_bounds__(256) relayout_kernel(const void *__restrict__ y_, void *__restrict__ z_,
                                                       const float2 *__restrict__ rot,
                                                       const float *__restrict__ inv_scale, int B, int fb, int Bs,
                                                       int QM, int K, int col) {
    using OutC = typename StoreT<ST>::c;
    using OutR = typename StoreT<ST>::r;
    constexpr int CB = (int)sizeof(OutR);          // bytes per component
    constexpr int SB = IQ ? 2 * CB : CB;           // bytes per sample
    unsigned char *zb = reinterpret_cast<unsigned char *>(z_);
    const int RB = fb * SB;
    __shared__ float2 tile[32][33];
    const int k0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int qm = blockIdx.y; qm < QM; qm += gridDim.y) {
    const float s = inv_scale ? inv_scale[qm] : 1.f;
    for (int bc = 0; bc < Bs; bc += 32) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int b = bc + ty + 8 * i, k = k0 + tx;
            float2 v = make_float2(0.f, 0.f);
            if (b < B && k < K) {
                const size_t idx = ((size_t)b * QM + qm) * (size_t)K + k;
                if (IQ) v = reinterpret_cast<const float2 *>(y_)[idx];
                else v.x = reinterpret_cast<const float *>(y_)[idx];
            }
            tile[ty + 8 * i][tx] = v;
        }
        __syncthreads();
        if constexpr (IQ && ST == ST_F32) {
            if (col && fb % 2 == 0) {
                // column order, float32 IQ: one thread writes a whole 16-byte piece
                // (re_2p, re_2p+1, im_2p, im_2p+1) of frames 2p, 2p + 1 of row k;
                // lanes run along k, so a warp writes 512 contiguous bytes
                for (int i = threadIdx.x; i < 16 * 32; i += 256) {
                    const int kl = i & 31, pp = i >> 5;
                    const int k = k0 + kl, b = bc + 2 * pp;  // bc and fb even: a pair never straddles a chunk
                    if (k < K && b < Bs) {
                        float2 v0 = tile[2 * pp][kl], v1 = tile[2 * pp + 1][kl];
                        if (rot) {
                            const float2 r = rot[k];
                            v0 = cmul(v0, r);
                            v1 = cmul(v1, r);
                        }
                        const int c = b / fb, j = b - c * fb;
                        unsigned char *blk = zb + ((size_t)c * QM + qm) * (size_t)K * RB;
                        *reinterpret_cast<float4 *>(blk + row_byte(k, 16 * (j >> 1), K, RB, true)) =
                            make_float4(v0.x * s, v1.x * s, v0.y * s, v1.y * s);
                    }
                }
                __syncthreads();
                continue;
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int kl = ty + 8 * i, k = k0 + kl, b = bc + tx;
            if (k < K && b < Bs) {
                float2 v = tile[tx][kl];
                const int c = b / fb, j = b - c * fb;
                unsigned char *blk = zb + ((size_t)c * QM + qm) * (size_t)K * RB;
                if (IQ) {
                    if (rot) v = cmul(v, rot[k]);
                    v.x *= s;
                    v.y *= s;
                    if (fb % 2 == 0) {
                        // pair-planar rows: re_{2p}, re_{2p+1}, im_{2p}, im_{2p+1}
                        const int rre = CB * (4 * (j >> 1) + (j & 1));
                        put(reinterpret_cast<OutR *>(blk + row_byte(k, rre, K, RB, col)), v.x);
                        put(reinterpret_cast<OutR *>(blk + row_byte(k, rre + 2 * CB, K, RB, col)), v.y);
                    } else {
                        put(reinterpret_cast<OutC *>(blk + row_byte(k, SB * j, K, RB, col)), v);
                    }
                } else {
                    put(reinterpret_cast<OutR *>(blk + row_byte(k, CB * j, K, RB, col)), v.x * s);
                }
            }
        }
        __syncthreads();
    }
    }
}

// Single frame: the layouts coincide; rotate / scale / convert elementwise.
template <bool IQ, int ST>
__global__ void __launch_bounds__(256) convert1_kernel(const void *__restrict__ y_, void *__restrict__ z_,
                                                       const float2 *__restrict__ rot,
                                                       const float *__restrict__ inv_scale, int QM, int K) {
    using OutC = typename StoreT<ST>::c;
    using OutR = typename StoreT<ST>::r;
    const size_t total = (size_t)QM * K;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % K);
        const float s = inv_scale ? inv_scale[i / K] : 1.f;
        if (IQ) {
            float2 v = reinterpret_cast<const float2 *>(y_)[i];
            if (rot) v = cmul(v, rot[k]);
            v.x *= s;
            v.y *= s;
            put(reinterpret_cast<OutC *>(z_) + i, v);
        } else {
            put(reinterpret_cast<OutR *>(z_) + i, reinterpret_cast<const float *>(y_)[i] * s);
        }
    }
}

template <bool IQ, int ST>
static cudaError_t relayout_dispatch(const void *y, void *z, const float2 *rot, const float *inv_scale, int B,
                                     int fb, int nch, int QM, int K, int col, cudaStream_t s) {
    const int Bs = fb * nch;
    if (Bs == 1) {
        if (col) return cudaErrorInvalidValue;  // single-sample rows are never read in column order
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const size_t total = (size_t)QM * K;
        const size_t cap = (size_t)sms * 32;
        const int blocks = (int)((total + 255) / 256 < cap ? (total + 255) / 256 : cap);
        convert1_kernel<IQ, ST><<<blocks, 256, 0, s>>>(y, z, rot, inv_scale, QM, K);
    } else {
        dim3 grid((K + 31) / 32, QM < 65535 ? QM : 65535);
        relayout_kernel<IQ, ST><<<grid, 256, 0, s>>>(y, z, rot, inv_scale, B, fb, Bs, QM, K, col);
    }
    return cudaSuccess;
}

cudaError_t launch_relayout(const void *y, void *z, const float2 *rot, const float *inv_scale, int iq, int store,
                            int B, int fb, int nch, int QM, int K, int col, cudaStream_t s) {
    cudaError_t e;
    if (iq) {
        if (store == ST_F32) e = relayout_dispatch<true, ST_F32>(y, z, rot, inv_scale, B, fb, nch, QM, K, col, s);
        else if (store == ST_F16) e = relayout_dispatch<true, ST_F16>(y, z, rot, inv_scale, B, fb, nch, QM, K, col, s);
        else if (store == ST_BF16) e = relayout_dispatch<true, ST_BF16>(y, z, rot, inv_scale, B, fb, nch, QM, K, col, s);
        else if (store == ST_E4M3) e = relayout_dispatch<true, ST_E4M3>(y, z, rot, inv_scale, B, fb, nch, QM, K, col, s);
        else e = relayout_dispatch<true, ST_E5M2>(y, z, rot, inv_scale, B, fb, nch, QM, K, col, s);
    } else {
        if (store == ST_F32) e = relayout_dispatch<false, ST_F32>(y, z, rot, inv_scale, B, fb, nch, QM, K, col, s);
        else if (store == ST_F16) e = relayout_dispatch<false, ST_F16>(y, z, rot, inv_scale, B, fb, nch, QM, K, col, s);
        else e = relayout_dispatch<false, ST_BF16>(y, z, rot, inv_scale, B, fb, nch, QM, K, col, s);
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

// ---------------------------------------------------------------------------
// reduce: one CTA, fixed order, float64
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(1024) reduce_kernel(const double *__restrict__ partial, long long n,
                                                      double *__restrict__ out) {
    double acc = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
    __shared__ double red[1024];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

cudaError_t launch_reduce(const double *partial, long long n, double *out, cudaStream_t s) {
    reduce_kernel<<<1, 1024, 0, s>>>(partial, n, out);
    return cudaGetLastError();
}

}  // namespace das
