// das_tile.cuh -- the voxel-tile kernel of the forward pass (Sec. 2, Eq. 2).
//
// One CTA owns one tile of 8 x 4 x 4 voxels (one voxel per thread) and a chunk
// of FB frames; every thread keeps FB complex (or real) accumulators in
// registers, so the per-(voxel, element, transmit) geometry is computed once
// and reused for all FB frames (the paper's B_tile reuse, Sec. 3.1, Alg. 1).
// The channel data are read in the batch-inner order z[q][m][k][b] (Sec. 3.2)
// so that the FB frames of one sample are contiguous and come in with 16-byte
// vector loads.  There are no atomics: each output is owned by one thread.
//
//  MODE_FWD   x_bn = sum_{q,m} w (1 - a) z[k] e^{i th a} + w a z[k+1] e^{-i th (1 - a)}
//  MODE_DC    the same sum of d/dc of each term (d tau_s / dc = -tau_s / c),
//             contracted with a cotangent and reduced to one partial per CTA
//  MODE_COUNT number of contributing terms, one partial per CTA
//
// Per element block of 128 elements, thread j evaluates element j's float64
// reference delay to the tile centre and a conservative aperture test for the
// whole tile; the elements that can contribute are compacted into shared
// memory and the CTA loops over them uniformly.
#pragma once

#include "das_internal.cuh"

namespace das {

template <bool IQ, int ST> struct SampleSize;
template <> struct SampleSize<true, ST_F32> { static constexpr int v = 8; };
template <> struct SampleSize<true, ST_F16> { static constexpr int v = 4; };
template <> struct SampleSize<true, ST_BF16> { static constexpr int v = 4; };
template <> struct SampleSize<false, ST_F32> { static constexpr int v = 4; };
template <> struct SampleSize<false, ST_F16> { static constexpr int v = 2; };
template <> struct SampleSize<false, ST_BF16> { static constexpr int v = 2; };
template <> struct SampleSize<true, ST_E4M3> { static constexpr int v = 2; };
template <> struct SampleSize<false, ST_E4M3> { static constexpr int v = 1; };
template <> struct SampleSize<true, ST_E5M2> { static constexpr int v = 2; };
template <> struct SampleSize<false, ST_E5M2> { static constexpr int v = 1; };

// Two 8-bit floats (E4M3 or E5M2, low byte first) as two floats.
template <int ST>
__device__ __forceinline__ float2 fp8x2_to_float2(uint32_t bits16) {
    static_assert(ST == ST_E4M3 || ST == ST_E5M2, "8-bit storage formats");
    const __half2_raw h =
        __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(bits16 & 0xffffu), ST == ST_E4M3 ? __NV_E4M3 : __NV_E5M2);
    return __half22float2(*reinterpret_cast<const __half2 *>(&h));
}

// FB consecutive samples of one row, loaded with the widest aligned vectors.
template <int FB, bool IQ, int ST> struct FrameRow {
    static constexpr int SZ = SampleSize<IQ, ST>::v;
    static constexpr int BYTES = FB * SZ;
    static constexpr bool HALFWORDS = (BYTES % 4) != 0;  // odd FB of 2-byte samples
    static constexpr int NW = HALFWORDS ? FB : BYTES / 4;
    static constexpr int VW = HALFWORDS ? 0 : (BYTES % 16 == 0) ? 4 : (BYTES % 8 == 0) ? 2 : 1;

    __device__ __forceinline__ static void load(const unsigned char *p, uint32_t (&w)[NW]) {
        if constexpr (HALFWORDS) {
#pragma unroll
            for (int i = 0; i < NW; ++i) w[i] = __ldg(reinterpret_cast<const unsigned short *>(p) + i);
        } else if constexpr (VW == 4) {
#pragma unroll
            for (int i = 0; i < NW / 4; ++i) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p) + i);
                w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
            }
        } else if constexpr (VW == 2) {
#pragma unroll
            for (int i = 0; i < NW / 2; ++i) {
                const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p) + i);
                w[2 * i] = v.x; w[2 * i + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < NW; ++i) w[i] = __ldg(reinterpret_cast<const unsigned int *>(p) + i);
        }
    }

    // Sample b as (re, im); im = 0 for RF.
    __device__ __forceinline__ static float2 get(const uint32_t (&w)[NW], int b) {
        if constexpr (IQ && ST == ST_F32) {
            return make_float2(__uint_as_float(w[2 * b]), __uint_as_float(w[2 * b + 1]));
        } else if constexpr (IQ && ST == ST_F16) {
            __half2 h;
            *reinterpret_cast<uint32_t *>(&h) = w[b];
            return __half22float2(h);
        } else if constexpr (IQ && ST == ST_BF16) {
            __nv_bfloat162 h;
            *reinterpret_cast<uint32_t *>(&h) = w[b];
            return __bfloat1622float2(h);
        } else if constexpr (IQ && (ST == ST_E4M3 || ST == ST_E5M2)) {
            const uint32_t bits = HALFWORDS ? w[b] : (w[b >> 1] >> (16 * (b & 1)));
            return fp8x2_to_float2<ST>(bits);
        } else if constexpr (!IQ && ST == ST_F32) {
            return make_float2(__uint_as_float(w[b]), 0.f);
        } else {
            const uint32_t bits = HALFWORDS ? w[b] : ((w[b >> 1] >> (16 * (b & 1))) & 0xffffu);
            const unsigned short hs = (unsigned short)bits;
            if constexpr (ST == ST_F16) return make_float2(__half2float(__ushort_as_half(hs)), 0.f);
            else return make_float2(__bfloat162float(__ushort_as_bfloat16(hs)), 0.f);
        }
    }
};

// How the tile kernels read sample rows from global memory.
//  LD_ROW  rows of FB samples stored contiguously (z[chunk][q][m][k][FB]),
//          128-bit loads;
//  LD_W256 the same rows with 256-bit loads;
//  LD_COL  the same bytes in column order: every row is cut into 16-byte
//          pieces and piece j of row k sits at j * (K * 16) + k * 16 inside
//          its (chunk, q, m) block, so the pieces of consecutive rows are
//          adjacent.  Lanes of a quarter-warp whose delays differ by a row or
//          two then read from one 128-byte line, where the row order puts
//          each distinct row in a line of its own (each line costs the L1 one
//          data-return wavefront).
enum LoadMode { LD_ROW = 0, LD_W256 = 1, LD_COL = 2 };

// Frames per register group of the global-load path, and whether the column
// order applies (rows and groups of whole 16-byte pieces).
template <int FB, bool IQ, int ST> struct ColShape {
    static constexpr int SZ = SampleSize<IQ, ST>::v;
    static constexpr int FG = (FB % 4 == 0 && (4 * SZ) % 16 == 0) ? 4 : FB;
    static constexpr bool ok = (FB * SZ) % 16 == 0 && (FG * SZ) % 16 == 0;
};

// 256-bit read-only global load (sm_100+), 32-byte aligned.
__device__ __forceinline__ void ldg256(const void *p, uint32_t *w) {
    asm volatile("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                 : "l"(p));
}

// Row of FB samples with 256-bit loads where the row is whole 32-byte vectors.
template <int FB, bool IQ, int ST, bool W256>
__device__ __forceinline__ void load_row(const unsigned char *p, uint32_t (&w)[FrameRow<FB, IQ, ST>::NW]) {
    using Row = FrameRow<FB, IQ, ST>;
    if constexpr (W256 && !Row::HALFWORDS && Row::BYTES % 32 == 0) {
#pragma unroll
        for (int i = 0; i < Row::NW / 8; ++i) ldg256(p + 32 * i, &w[8 * i]);
    } else {
        Row::load(p, w);
    }
}

// FB samples of one row in column order: 16-byte piece i at p + i * cs.
template <int FB, bool IQ, int ST>
__device__ __forceinline__ void load_col(const unsigned char *p, size_t cs, uint32_t (&w)[FrameRow<FB, IQ, ST>::NW]) {
    using Row = FrameRow<FB, IQ, ST>;
    static_assert(!Row::HALFWORDS && Row::BYTES % 16 == 0, "column order needs whole 16-byte pieces");
#pragma unroll
    for (int i = 0; i < Row::NW / 4; ++i) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p + i * cs));
        w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
    }
}

// FB frame accumulators of one voxel.  With an even FB the rows are
// pair-planar (IQ) or naturally paired (RF) and two frames are updated by one
// packed float32 FMA (__ffma2_rn); with an odd FB the frames are updated one
// by one from interleaved (re, im) samples.
template <int FB, bool IQ, int ST> struct FrameAcc {
    static constexpr bool PAIR = (FB % 2) == 0;
    using Row = FrameRow<FB, IQ, ST>;
    static constexpr int NP = PAIR ? FB / 2 : 1;
    static constexpr int NS = PAIR ? 1 : FB;
    float2 re2[NP], im2[NP];
    float re1[NS], im1[NS];

    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int p = 0; p < NP; ++p) re2[p] = im2[p] = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < NS; ++b) re1[b] = im1[b] = 0.f;
    }

    // (re, im) of frame pair p: two float2 holding frames 2p and 2p+1
    __device__ __forceinline__ static void pair(const uint32_t *w, int p, float2 &re, float2 &im) {
        if constexpr (IQ && ST == ST_F32) {
            re = make_float2(__uint_as_float(w[4 * p]), __uint_as_float(w[4 * p + 1]));
            im = make_float2(__uint_as_float(w[4 * p + 2]), __uint_as_float(w[4 * p + 3]));
        } else if constexpr (IQ && ST == ST_F16) {
            __half2 a, b;
            *reinterpret_cast<uint32_t *>(&a) = w[2 * p];
            *reinterpret_cast<uint32_t *>(&b) = w[2 * p + 1];
            re = __half22float2(a);
            im = __half22float2(b);
        } else if constexpr (IQ && ST == ST_BF16) {
            __nv_bfloat162 a, b;
            *reinterpret_cast<uint32_t *>(&a) = w[2 * p];
            *reinterpret_cast<uint32_t *>(&b) = w[2 * p + 1];
            re = __bfloat1622float2(a);
            im = __bfloat1622float2(b);
        } else if constexpr (IQ && (ST == ST_E4M3 || ST == ST_E5M2)) {
            re = fp8x2_to_float2<ST>(w[p]);        // bytes re_2p, re_2p+1
            im = fp8x2_to_float2<ST>(w[p] >> 16);  // bytes im_2p, im_2p+1
        } else if constexpr (ST == ST_F32) {
            re = make_float2(__uint_as_float(w[2 * p]), __uint_as_float(w[2 * p + 1]));
        } else if constexpr (ST == ST_F16) {
            __half2 a;
            *reinterpret_cast<uint32_t *>(&a) = w[p];
            re = __half22float2(a);
        } else {
            __nv_bfloat162 a;
            *reinterpret_cast<uint32_t *>(&a) = w[p];
            re = __bfloat1622float2(a);
        }
    }

    // acc += c0 * tap0 + c1 * tap1 for frames [g0, g0 + G) of words w0, w1
    // (w holds those frames only, starting at frame g0)
    template <int G>
    __device__ __forceinline__ void add(int g0, const uint32_t *w0, const uint32_t *w1, float c0r, float c0i,
                                        float c1r, float c1i) {
        if constexpr (PAIR) {
            const float2 C0R = make_float2(c0r, c0r), C0I = make_float2(c0i, c0i);
            const float2 N0I = make_float2(-c0i, -c0i), C1R = make_float2(c1r, c1r);
            const float2 C1I = make_float2(c1i, c1i), N1I = make_float2(-c1i, -c1i);
#pragma unroll
            for (int p = 0; p < G / 2; ++p) {
                float2 zr0, zi0, zr1, zi1;
                pair(w0, p, zr0, zi0);
                pair(w1, p, zr1, zi1);
                const int q = g0 / 2 + p;
                if constexpr (IQ) {
                    re2[q] = __ffma2_rn(C0R, zr0, re2[q]);
                    re2[q] = __ffma2_rn(N0I, zi0, re2[q]);
                    re2[q] = __ffma2_rn(C1R, zr1, re2[q]);
                    re2[q] = __ffma2_rn(N1I, zi1, re2[q]);
                    im2[q] = __ffma2_rn(C0R, zi0, im2[q]);
                    im2[q] = __ffma2_rn(C0I, zr0, im2[q]);
                    im2[q] = __ffma2_rn(C1R, zi1, im2[q]);
                    im2[q] = __ffma2_rn(C1I, zr1, im2[q]);
                } else {
                    re2[q] = __ffma2_rn(C0R, zr0, re2[q]);
                    re2[q] = __ffma2_rn(C1R, zr1, re2[q]);
                }
            }
        } else {
            using RowG = FrameRow<G, IQ, ST>;
#pragma unroll
            for (int b = 0; b < G; ++b) {
                const float2 z0 = RowG::get(*reinterpret_cast<const uint32_t(*)[RowG::NW]>(w0), b);
                const float2 z1 = RowG::get(*reinterpret_cast<const uint32_t(*)[RowG::NW]>(w1), b);
                const int f = g0 + b;
                if constexpr (IQ) {
                    re1[f] = fmaf(c0r, z0.x, fmaf(-c0i, z0.y, fmaf(c1r, z1.x, fmaf(-c1i, z1.y, re1[f]))));
                    im1[f] = fmaf(c0r, z0.y, fmaf(c0i, z0.x, fmaf(c1r, z1.y, fmaf(c1i, z1.x, im1[f]))));
                } else {
                    re1[f] = fmaf(c0r, z0.x, fmaf(c1r, z1.x, re1[f]));
                }
            }
        }
    }

    // acc += c0 * tap0 + c1 * tap1 + c2 * tap2 (three rows; even FB, IQ):
    // the second voxel of a thread pair, whose two taps sit at two of three
    // rows loaded once for both voxels (das_tile_pair.cuh)
    template <int G>
    __device__ __forceinline__ void add3(int g0, const uint32_t *w0, const uint32_t *w1, const uint32_t *w2,
                                         float c0r, float c0i, float c1r, float c1i, float c2r, float c2i) {
        static_assert(PAIR && IQ, "three-row updates are for pair-planar IQ rows");
        const float2 C0R = make_float2(c0r, c0r), C0I = make_float2(c0i, c0i), N0I = make_float2(-c0i, -c0i);
        const float2 C1R = make_float2(c1r, c1r), C1I = make_float2(c1i, c1i), N1I = make_float2(-c1i, -c1i);
        const float2 C2R = make_float2(c2r, c2r), C2I = make_float2(c2i, c2i), N2I = make_float2(-c2i, -c2i);
#pragma unroll
        for (int p = 0; p < G / 2; ++p) {
            float2 zr0, zi0, zr1, zi1, zr2, zi2;
            pair(w0, p, zr0, zi0);
            pair(w1, p, zr1, zi1);
            pair(w2, p, zr2, zi2);
            const int q = g0 / 2 + p;
            re2[q] = __ffma2_rn(C0R, zr0, re2[q]);
            re2[q] = __ffma2_rn(N0I, zi0, re2[q]);
            re2[q] = __ffma2_rn(C1R, zr1, re2[q]);
            re2[q] = __ffma2_rn(N1I, zi1, re2[q]);
            re2[q] = __ffma2_rn(C2R, zr2, re2[q]);
            re2[q] = __ffma2_rn(N2I, zi2, re2[q]);
            im2[q] = __ffma2_rn(C0R, zi0, im2[q]);
            im2[q] = __ffma2_rn(C0I, zr0, im2[q]);
            im2[q] = __ffma2_rn(C1R, zi1, im2[q]);
            im2[q] = __ffma2_rn(C1I, zr1, im2[q]);
            im2[q] = __ffma2_rn(C2R, zi2, im2[q]);
            im2[q] = __ffma2_rn(C2I, zr2, im2[q]);
        }
    }

    __device__ __forceinline__ float re(int b) const {
        if constexpr (PAIR) return (b & 1) ? re2[b >> 1].y : re2[b >> 1].x;
        else return re1[b];
    }
    __device__ __forceinline__ float im(int b) const {
        if constexpr (PAIR) return (b & 1) ? im2[b >> 1].y : im2[b >> 1].x;
        else return im1[b];
    }
};

// Resident CTAs per SM asked of the compiler: wide rows of float32 IQ samples
// (16 or more frames, 8 bytes each) keep 3 CTAs, which avoids spilling.
template <int FB, int SZ = 4> struct TileOcc {
    static constexpr int v = FB <= 4 ? 6 : FB <= 12 ? 5 : (SZ >= 8 ? 3 : 4);
};

// One (tile, frame chunk) of one plan with rows read from global memory;
// `smem` is the CTA's dynamic shared memory (tile_smem_bytes).  Called by
// tile_kernel (one launch per plan) and by the persistent batch kernel.
template <int FB, bool IQ, int ST, int MODE, int LD = LD_ROW>
__device__ __forceinline__ void tile_body(const TileArgs &A, const long long tile, const int chunk,
                                          unsigned char *smem, const unsigned grid_x) {
    using Row = FrameRow<FB, IQ, ST>;
    constexpr int SZ = Row::SZ;
    const int Q = A.Q;
    const bool has_w = A.w_tx != nullptr;
    float4 *s_eg = reinterpret_cast<float4 *>(smem);                  // [128] (G, |G|)
    float4 *s_en = s_eg + TILE_N;                                       // [128] (normal, rf)
    float *s_t = reinterpret_cast<float *>(s_en + TILE_N);             // [Q][128]
    float *s_w = s_t + Q * TILE_N;                                      // [Q][128] when has_w
    int *s_erb = reinterpret_cast<int *>(s_w + (has_w ? Q * TILE_N : 0));  // [128]
    int *s_em = s_erb + TILE_N;                                         // [128]
    int *s_tb = s_em + TILE_N;                                          // [Q]
    int *s_cnt = s_tb + Q;                                              // [5]

    const int tid = threadIdx.x;
    const int b0 = chunk * FB;
    const GridDesc &g = A.g;
    const int tx = (int)(tile % g.tiles_x);
    const int ty = (int)((tile / g.tiles_x) % g.tiles_y);
    const int tz = (int)(tile / ((long long)g.tiles_x * g.tiles_y));
    int lx, ly, lz;
    lane_offset(tid, lx, ly, lz);
    const int ix = tx * TILE_X + lx, iy = ty * TILE_Y + ly, iz = tz * TILE_Z + lz;
    const bool valid = ix < g.nx && iy < g.ny && iz < g.nz;
    const long long n = ((long long)iz * g.ny + iy) * g.nx + ix;
    double p0x, p0y, p0z;
    tile_centre(g, tx, ty, tz, p0x, p0y, p0z);
    const float dx = (float)(g.sx * (lx - 0.5 * (TILE_X - 1)));
    const float dy = (float)(g.sy * (ly - 0.5 * (TILE_Y - 1)));
    const float dz = (float)(g.sz * (lz - 0.5 * (TILE_Z - 1)));
    const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));

    __syncthreads();  // a previous body call on this CTA is done with shared memory
    for (int q = 0; q < Q; ++q) {
        s_t[q * TILE_N + tid] = A.tx_t[(tile * Q + q) * TILE_N + tid];
        if (has_w) s_w[q * TILE_N + tid] = A.w_tx[(tile * Q + q) * TILE_N + tid];
    }
    for (int q = tid; q < Q; q += TILE_N) s_tb[q] = A.tx_tb[tile * Q + q];

    FrameAcc<FB, IQ, ST> acc;
    acc.zero();
    long long count = 0;

    const int lane = tid & 31, warp = tid >> 5;
    for (int m0 = 0; m0 < A.M; m0 += TILE_N) {
        __syncthreads();  // previous block's records are no longer read
        const int m = m0 + tid;
        bool cand = false;
        float4 eg = make_float4(0.f, 0.f, 0.f, 0.f), en = eg;
        int rb = 0;
        if (m < A.M) {
            const double rx = A.elem_pos[3 * m], ry = A.elem_pos[3 * m + 1], rz = A.elem_pos[3 * m + 2];
            const double Gx = p0x - rx, Gy = p0y - ry, Gz = p0z - rz;
            const double D0 = sqrt(Gx * Gx + Gy * Gy + Gz * Gz);
            const double R0 = A.ad * D0;
            const double Rf = floor(R0);
            rb = (int)Rf;
            const float4 nn = A.elem_nrm[m];
            eg = make_float4((float)Gx, (float)Gy, (float)Gz, (float)D0);
            en = make_float4(nn.x, nn.y, nn.z, (float)(R0 - Rf));
            cand = true;
            if (A.thr >= 0.f) {
                const float z0 = eg.x * nn.x + eg.y * nn.y + eg.z * nn.z;
                const float cx = eg.y * nn.z - eg.z * nn.y, cy = eg.z * nn.x - eg.x * nn.z,
                            cz = eg.x * nn.y - eg.y * nn.x;
                const float rho0 = sqrtf(cx * cx + cy * cy + cz * cz);
                const float zmax = z0 + A.tile_radius;
                const float rmin = fmaxf(rho0 - A.tile_radius, 0.f);
                cand = (zmax > 0.f) && (rmin * rmin <= A.thr * zmax * zmax * 1.001f);
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, cand);
        if (lane == 0) s_cnt[warp] = __popc(bal);
        __syncthreads();
        int off = 0;
        for (int w = 0; w < warp; ++w) off += s_cnt[w];
        if (cand) {
            const int idx = off + __popc(bal & ((1u << lane) - 1u));
            s_eg[idx] = eg;
            s_en[idx] = en;
            s_erb[idx] = rb;
            s_em[idx] = m;
        }
        const int total = s_cnt[0] + s_cnt[1] + s_cnt[2] + s_cnt[3];
        __syncthreads();

        for (int j = 0; j < total; ++j) {
            const float4 G = s_eg[j];
            const float4 Nn = s_en[j];
            const float ex = G.x + dx, ey = G.y + dy, ez = G.z + dz;
            bool inside = valid;
            if (A.thr >= 0.f) {
                const float zax = fmaf(ex, Nn.x, fmaf(ey, Nn.y, ez * Nn.z));
                const float cx = fmaf(ey, Nn.z, -ez * Nn.y), cy = fmaf(ez, Nn.x, -ex * Nn.z),
                            cz = fmaf(ex, Nn.y, -ey * Nn.x);
                const float rho2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
                inside = inside && (zax > 0.f) && (rho2 <= A.thr * zax * zax);
            }
            if (!inside) continue;
            const int Rb = s_erb[j];
            const int mm = s_em[j];
            const float d = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
            const float num = fmaf(2.f, fmaf(G.x, dx, fmaf(G.y, dy, G.z * dz)), dd);
            const float r = Nn.w + A.a * __fdividef(num, d + G.w);
            // chunk-major blocks of K rows: z[chunk][q][m][K rows of FB samples]
            const unsigned char *zrow = reinterpret_cast<const unsigned char *>(A.z) +
                                        (((size_t)chunk * Q * A.M + mm) * A.K) * (size_t)(FB * SZ);
            const size_t qstride = (size_t)A.M * A.K * (FB * SZ);
            const size_t cs = (size_t)A.K * 16;  // LD_COL: bytes between the pieces of a row
#pragma unroll 2
            for (int q = 0; q < Q; ++q) {
                const float f = r + s_t[q * TILE_N + tid];
                const float fl = floorf(f);
                const float al = f - fl;
                const int k = s_tb[q] + Rb + (int)fl;
                if ((unsigned)k > (unsigned)(A.K - 2)) continue;
                if constexpr (MODE == MODE_COUNT) {
                    ++count;
                    continue;
                }
                float w = has_w ? s_w[q * TILE_N + tid] : 1.f;
                if (ST != ST_F32) w *= __ldg(A.scale + (size_t)q * A.M + mm);
                float c0r, c0i = 0.f, c1r, c1i = 0.f;
                if constexpr (IQ) {
                    float sn, cs;
                    __sincosf(A.theta * (al - 0.5f), &sn, &cs);
                    const float uhr = cs * A.hr - sn * A.hi, uhi = cs * A.hi + sn * A.hr;  // e^{i th a}
                    const float ubr = cs * A.hr + sn * A.hi, ubi = sn * A.hr - cs * A.hi;  // e^{-i th (1-a)}
                    if constexpr (MODE == MODE_FWD) {
                        const float w0 = w * (1.f - al), w1 = w * al;
                        c0r = w0 * uhr; c0i = w0 * uhi;
                        c1r = w1 * ubr; c1i = w1 * ubi;
                    } else {
                        const float s = -w * ((float)k + al) * (float)A.inv_c;
                        const float a0 = A.theta * (1.f - al), a1 = A.theta * al;
                        c0r = s * (-uhr - a0 * uhi); c0i = s * (a0 * uhr - uhi);
                        c1r = s * (ubr - a1 * ubi); c1i = s * (ubi + a1 * ubr);
                    }
                } else {
                    if constexpr (MODE == MODE_FWD) {
                        c0r = w * (1.f - al);
                        c1r = w * al;
                    } else {
                        const float s = -w * ((float)k + al) * (float)A.inv_c;
                        c0r = -s;
                        c1r = s;
                    }
                }
                constexpr bool COL = LD == LD_COL;
                constexpr int RSTEP = COL ? 16 : FB * SZ;  // bytes from row k to row k + 1
                const unsigned char *p0 = zrow + q * qstride + (size_t)k * RSTEP;
                const unsigned char *p1 = p0 + RSTEP;
                // rows k and k+1 in groups of FG frames (fewer live registers)
                constexpr int FG = LD == LD_W256 ? FB : ColShape<FB, IQ, ST>::FG;
                static_assert(!COL || ColShape<FB, IQ, ST>::ok, "column order needs whole 16-byte pieces");
                using RowG = FrameRow<FG, IQ, ST>;
#pragma unroll
                for (int bg = 0; bg < FB; bg += FG) {
                    uint32_t w0[RowG::NW], w1[RowG::NW];
                    if constexpr (COL) {
                        const size_t off = (size_t)(bg * SZ / 16) * cs;
                        load_col<FG, IQ, ST>(p0 + off, cs, w0);
                        load_col<FG, IQ, ST>(p1 + off, cs, w1);
                    } else {
                        load_row<FG, IQ, ST, LD == LD_W256>(p0 + bg * SZ, w0);
                        load_row<FG, IQ, ST, LD == LD_W256>(p1 + bg * SZ, w1);
                    }
                    acc.template add<FG>(bg, w0, w1, c0r, c0i, c1r, c1i);
                }
            }
        }
    }

    if constexpr (MODE == MODE_FWD) {
        if (valid) {
#pragma unroll
            for (int b = 0; b < FB; ++b) {
                if (b0 + b < A.B) {
                    const size_t o = (size_t)(b0 + b) * g.n_voxels + n;
                    if constexpr (IQ) reinterpret_cast<float2 *>(A.x)[o] = make_float2(acc.re(b), acc.im(b));
                    else reinterpret_cast<float *>(A.x)[o] = acc.re(b);
                }
            }
        }
    } else {
        double v = 0.0;
        if constexpr (MODE == MODE_COUNT) {
            v = (double)count;
        } else if (valid) {
#pragma unroll
            for (int b = 0; b < FB; ++b) {
                if (b0 + b < A.B) {
                    const size_t o = (size_t)(b0 + b) * g.n_voxels + n;
                    if constexpr (IQ) {
                        const float2 gv = reinterpret_cast<const float2 *>(A.gx)[o];
                        v += (double)gv.x * acc.re(b) + (double)gv.y * acc.im(b);
                    } else {
                        v += (double)reinterpret_cast<const float *>(A.gx)[o] * acc.re(b);
                    }
                }
            }
        }
        double *red = reinterpret_cast<double *>(s_eg);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();  // every warp is done reading the element records red reuses
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < TILE_N / 32; ++w) s += red[w];
            A.partial[(size_t)chunk * grid_x + tile] = s;
        }
    }
}

template <int FB, bool IQ, int ST, int MODE, int LD = LD_ROW>
__global__ void __launch_bounds__(TILE_N, (TileOcc<FB, SampleSize<IQ, ST>::v>::v)) tile_kernel(const TileArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    tile_body<FB, IQ, ST, MODE, LD>(A, blockIdx.x, blockIdx.y, smem, gridDim.x);
}

inline size_t tile_smem_bytes(int Q, bool has_w) {
    return sizeof(float4) * 2 * TILE_N + sizeof(float) * (size_t)Q * TILE_N * (has_w ? 2 : 1) +
           sizeof(int) * (2 * TILE_N + Q + 5);
}

template <int FB, bool IQ, int ST, int MODE, int LD = LD_ROW>
cudaError_t launch_tile_t(const TileArgs &A, int n_chunks, cudaStream_t s) {
    const size_t smem = tile_smem_bytes(A.Q, A.w_tx != nullptr);
    auto kern = tile_kernel<FB, IQ, ST, MODE, LD>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)n_tiles(A.g), (unsigned)n_chunks);
    kern<<<grid, TILE_N, smem, s>>>(A);
    return cudaGetLastError();
}

}  // namespace das
