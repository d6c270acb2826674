// das_tile_pair.cuh -- the forward tile kernel with two voxels per thread that
// share sample rows (Sec. 2, Eq. 2; float32 IQ storage in column order).
//
// The float32 tile kernel (das_tile.cuh) is bound by the L1 data-return
// path: every (voxel, element, transmit) term brings two sample rows of FB
// frames into registers, 16 bytes per frame for 8 FMAs, while the L1 returns
// 128 bytes per clock per SM against 128 FMA lanes.  Voxels one step apart
// along x have delays less than about one sample apart (the lateral slope of
// the delay is below one sample per 0.1 mm voxel inside an f-number-1
// aperture), so their taps fall on two or three consecutive rows.  Here one
// thread owns such a pair and loads three rows once for both: 1.5 rows per
// voxel instead of 2.
//
// Block: two tiles side by side along x (16 x 4 x 4 voxels), 128 threads.
// Warp w is the z-layer w; quarter-warp qd covers the x-half qd & 1 and the
// y rows 2 (qd >> 1), +1; lane w8 of a quarter owns voxels x = 2 (w8 & 3) and
// x + 1 of that half, y = (w8 >> 2) + 2 (qd >> 1).  The per-tile transmit
// tables of the prepare kernel serve both tiles; the float64 receive
// reference of each element is taken at the centre of the block.
//
// Per (element, transmit) the thread forms k_A and k_B.  Voxel A reads rows
// k0 = k_A, k0 + 1 with its two tap weights; voxel B reads the same two rows
// plus a third one, row k0 + 2 when k_B = k_A + 1 or row k0 - 1 when
// k_B = k_A - 1, with three weights of which one is zero (k_B = k_A: the
// third row is not loaded).  When only one voxel contributes it is the
// reference; when |k_B - k_A| >= 2 (outside the aperture's slopes, rare) B
// loads its own two rows.
#pragma once

#include "das_tile.cuh"

namespace das {

// Voxels of lane l of a pair block: tile half h, x0 (and x0 + 1) inside that
// tile, y, z.
__host__ __device__ inline void pair_lane(int l, int &h, int &x0, int &ly, int &lz) {
    const int w8 = l & 7, qd = (l >> 3) & 3;
    h = qd & 1;
    x0 = 2 * (w8 & 3);
    ly = (w8 >> 2) | ((qd >> 1) << 1);
    lz = l >> 5;
}

// Lane of voxel (lx, ly, lz) of a tile in the order of lane_offset (its inverse).
__host__ __device__ inline int tile_lane(int lx, int ly, int lz) {
    return ((lx & 3) | ((ly & 1) << 2)) | (((lx >> 2) | ((ly >> 1) << 1)) << 3) | (lz << 5);
}

inline size_t pair_smem_bytes(int Q, bool has_w) {
    return sizeof(float4) * 2 * TILE_N + sizeof(float) * (size_t)2 * Q * TILE_N * (has_w ? 2 : 1) +
           sizeof(int) * (2 * TILE_N + 2 * Q + 5);
}

// Complex tap weights of one term (forward): w (1 - a) e^{i th a} on row k and
// w a e^{-i th (1 - a)} on row k + 1 (pre-rotated samples; das_internal.cuh).
__device__ __forceinline__ void tap_weights(const TileArgs &A, float w, float al, float &c0r, float &c0i, float &c1r,
                                            float &c1i) {
    float sn, cs;
    __sincosf(A.theta * (al - 0.5f), &sn, &cs);
    const float uhr = cs * A.hr - sn * A.hi, uhi = cs * A.hi + sn * A.hr;  // e^{i th a}
    const float ubr = cs * A.hr + sn * A.hi, ubi = sn * A.hr - cs * A.hi;  // e^{-i th (1-a)}
    const float w0 = w * (1.f - al), w1 = w * al;
    c0r = w0 * uhr; c0i = w0 * uhi;
    c1r = w1 * ubr; c1i = w1 * ubi;
}

template <int FB, int ST>
__global__ void __launch_bounds__(TILE_N, 3) pair_kernel(const TileArgs A) {
    constexpr bool IQ = true;
    using Shape = ColShape<FB, IQ, ST>;
    static_assert(FB % 2 == 0 && Shape::ok, "pair kernel: pair-planar rows of whole 16-byte pieces");
    constexpr int SZ = Shape::SZ;
    constexpr int FG = 16 / SZ;  // frames per register group: one 16-byte piece per row (fewer live registers)
    static_assert(FB % FG == 0, "frame groups of whole pieces");
    using RowG = FrameRow<FG, IQ, ST>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int Q = A.Q;
    const bool has_w = A.w_tx != nullptr;
    float4 *s_eg = reinterpret_cast<float4 *>(smem);                    // [128] (G, |G|)
    float4 *s_en = s_eg + TILE_N;                                         // [128] (normal, rf)
    float *s_t = reinterpret_cast<float *>(s_en + TILE_N);               // [2][Q][128]
    float *s_w = s_t + 2 * Q * TILE_N;                                    // [2][Q][128] when has_w
    int *s_erb = reinterpret_cast<int *>(s_w + (has_w ? 2 * Q * TILE_N : 0));  // [128]
    int *s_em = s_erb + TILE_N;                                           // [128]
    int *s_tb = s_em + TILE_N;                                            // [2][Q]
    int *s_cnt = s_tb + 2 * Q;                                            // [5]

    const GridDesc &g = A.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int pairs_x = (g.tiles_x + 1) >> 1;
    const long long pb = blockIdx.x;
    const int chunk = blockIdx.y;
    const int b0 = chunk * FB;
    const int px = (int)(pb % pairs_x);
    const int ty = (int)((pb / pairs_x) % g.tiles_y);
    const int tz = (int)(pb / ((long long)pairs_x * g.tiles_y));
    const int tx0 = 2 * px;
    const bool has2 = tx0 + 1 < g.tiles_x;
    const long long tile0 = ((long long)tz * g.tiles_y + ty) * g.tiles_x + tx0;

    int h, x0, ly, lz;
    pair_lane(tid, h, x0, ly, lz);
    const int ixA = (tx0 + h) * TILE_X + x0, iy = ty * TILE_Y + ly, iz = tz * TILE_Z + lz;
    const bool rowok = (h == 0 || has2) && iy < g.ny && iz < g.nz;
    const bool validA = rowok && ixA < g.nx, validB = rowok && ixA + 1 < g.nx;
    const int laneA = tile_lane(x0, ly, lz), laneB = tile_lane(x0 + 1, ly, lz);
    const long long nA = ((long long)iz * g.ny + iy) * g.nx + ixA;
    // block centre: between the two tiles along x
    const double p0x = g.ox + g.sx * (tx0 * TILE_X + (TILE_X - 0.5));
    const double p0y = g.oy + g.sy * (ty * TILE_Y + 0.5 * (TILE_Y - 1));
    const double p0z = g.oz + g.sz * (tz * TILE_Z + 0.5 * (TILE_Z - 1));
    const float dxA = (float)(g.sx * (h * TILE_X + x0 - (TILE_X - 0.5)));
    const float dxB = (float)(g.sx * (h * TILE_X + x0 + 1 - (TILE_X - 0.5)));
    const float dy = (float)(g.sy * (ly - 0.5 * (TILE_Y - 1)));
    const float dz = (float)(g.sz * (lz - 0.5 * (TILE_Z - 1)));
    const float ddA = fmaf(dxA, dxA, fmaf(dy, dy, dz * dz));
    const float ddB = fmaf(dxB, dxB, fmaf(dy, dy, dz * dz));
    // block radius (half diagonal of its voxel centres) for the element pre-test
    const float brad = (float)(sqrt((TILE_X - 0.5) * (TILE_X - 0.5) * g.sx * g.sx +
                                    0.25 * (TILE_Y - 1) * (TILE_Y - 1) * g.sy * g.sy +
                                    0.25 * (TILE_Z - 1) * (TILE_Z - 1) * g.sz * g.sz) * (1.0 + 1e-4) + 1e-9);

    for (int hh = 0; hh < 2; ++hh) {
        const bool ok = hh == 0 || has2;
        const long long t = tile0 + hh;
        for (int q = 0; q < Q; ++q) {
            s_t[(hh * Q + q) * TILE_N + tid] = ok ? A.tx_t[(t * Q + q) * TILE_N + tid] : 0.f;
            if (has_w) s_w[(hh * Q + q) * TILE_N + tid] = ok ? A.w_tx[(t * Q + q) * TILE_N + tid] : 0.f;
        }
        for (int q = tid; q < Q; q += TILE_N) s_tb[hh * Q + q] = ok ? A.tx_tb[t * Q + q] : 0;
    }

    FrameAcc<FB, IQ, ST> accA, accB;
    accA.zero();
    accB.zero();
    const float *tA = s_t + h * Q * TILE_N + laneA;
    const float *tB = s_t + h * Q * TILE_N + laneB;
    const int *tbh = s_tb + h * Q;
    const size_t cs = (size_t)A.K * 16;  // bytes between the pieces of a row (column order)
    const size_t qstride = (size_t)A.M * A.K * (FB * SZ);

    for (int m0 = 0; m0 < A.M; m0 += TILE_N) {
        __syncthreads();  // previous block's records are no longer read (and the tables are loaded)
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
                const float zmax = z0 + brad;
                const float rmin = fmaxf(rho0 - brad, 0.f);
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
            const float exA = G.x + dxA, exB = G.x + dxB, ey = G.y + dy, ez = G.z + dz;
            bool inA = validA, inB = validB;
            if (A.thr >= 0.f) {
                const float cyz = fmaf(ey, Nn.z, -ez * Nn.y);  // shared by both voxels
                const float zA = fmaf(exA, Nn.x, fmaf(ey, Nn.y, ez * Nn.z));
                const float zB = fmaf(exB, Nn.x, fmaf(ey, Nn.y, ez * Nn.z));
                const float cyA = fmaf(ez, Nn.x, -exA * Nn.z), czA = fmaf(exA, Nn.y, -ey * Nn.x);
                const float cyB = fmaf(ez, Nn.x, -exB * Nn.z), czB = fmaf(exB, Nn.y, -ey * Nn.x);
                const float rA2 = fmaf(cyz, cyz, fmaf(cyA, cyA, czA * czA));
                const float rB2 = fmaf(cyz, cyz, fmaf(cyB, cyB, czB * czB));
                inA = inA && (zA > 0.f) && (rA2 <= A.thr * zA * zA);
                inB = inB && (zB > 0.f) && (rB2 <= A.thr * zB * zB);
            }
            if (!inA && !inB) continue;
            const int Rb = s_erb[j];
            const int mm = s_em[j];
            const float gdyz = fmaf(G.y, dy, G.z * dz);
            const float dA = sqrtf(fmaf(exA, exA, fmaf(ey, ey, ez * ez)));
            const float dB = sqrtf(fmaf(exB, exB, fmaf(ey, ey, ez * ez)));
            const float rA = Nn.w + A.a * __fdividef(fmaf(2.f, fmaf(G.x, dxA, gdyz), ddA), dA + G.w);
            const float rB = Nn.w + A.a * __fdividef(fmaf(2.f, fmaf(G.x, dxB, gdyz), ddB), dB + G.w);
            const unsigned char *zq = reinterpret_cast<const unsigned char *>(A.z) +
                                      (((size_t)chunk * Q * A.M + mm) * A.K) * (size_t)(FB * SZ);
#pragma unroll 1
            for (int q = 0; q < Q; ++q) {
                const float fA = rA + tA[q * TILE_N], fB = rB + tB[q * TILE_N];
                const float flA = floorf(fA), flB = floorf(fB);
                const float alA = fA - flA, alB = fB - flB;
                const int kbase = tbh[q] + Rb;
                const int kA = kbase + (int)flA, kB = kbase + (int)flB;
                const bool okA = inA && (unsigned)kA <= (unsigned)(A.K - 2);
                const bool okB = inB && (unsigned)kB <= (unsigned)(A.K - 2);
                if (!okA && !okB) continue;
                float c0r = 0.f, c0i = 0.f, c1r = 0.f, c1i = 0.f;  // voxel A
                float e0r = 0.f, e0i = 0.f, e1r = 0.f, e1i = 0.f;  // voxel B
                if (okA) {
                    const float w = has_w ? s_w[(h * Q + q) * TILE_N + laneA] : 1.f;
                    tap_weights(A, w, alA, c0r, c0i, c1r, c1i);
                }
                if (okB) {
                    const float w = has_w ? s_w[(h * Q + q) * TILE_N + laneB] : 1.f;
                    tap_weights(A, w, alB, e0r, e0i, e1r, e1i);
                }
                // reference rows k0, k0 + 1: voxel A's, or B's when A does not contribute
                const int k0 = okA ? kA : kB;
                const int dk = okA && okB ? kB - kA : 0;
                const unsigned char *p0 = zq + q * qstride + (size_t)k0 * 16;
                if (dk >= -1 && dk <= 1) {
                    // B's three weights over (row k0, row k0 + 1, third row)
                    const bool up = dk == 1, down = dk == -1;
                    const float b0r = up ? 0.f : (down ? e1r : e0r), b0i = up ? 0.f : (down ? e1i : e0i);
                    const float b1r = up ? e0r : (down ? 0.f : e1r), b1i = up ? e0i : (down ? 0.f : e1i);
                    const float b2r = up ? e1r : (down ? e0r : 0.f), b2i = up ? e1i : (down ? e0i : 0.f);
                    const bool third = up || down;
                    const unsigned char *p2 = up ? p0 + 32 : p0 - 16;
                    // A's weights on the reference rows are zero when only B contributes
#pragma unroll
                    for (int bg = 0; bg < FB; bg += FG) {
                        const size_t off = (size_t)(bg * SZ / 16) * cs;
                        uint32_t w0[RowG::NW], w1[RowG::NW], w2[RowG::NW];
                        load_col<FG, IQ, ST>(p0 + off, cs, w0);
                        load_col<FG, IQ, ST>(p0 + 16 + off, cs, w1);
                        if (third) {
                            load_col<FG, IQ, ST>(p2 + off, cs, w2);
                        } else {
#pragma unroll
                            for (int i = 0; i < RowG::NW; ++i) w2[i] = 0u;
                        }
                        accA.template add<FG>(bg, w0, w1, c0r, c0i, c1r, c1i);
                        accB.template add3<FG>(bg, w0, w1, w2, b0r, b0i, b1r, b1i, b2r, b2i);
                    }
                } else {
                    // delays two or more rows apart: each voxel reads its own two rows
                    const unsigned char *pB = zq + q * qstride + (size_t)kB * 16;
#pragma unroll
                    for (int bg = 0; bg < FB; bg += FG) {
                        const size_t off = (size_t)(bg * SZ / 16) * cs;
                        uint32_t w0[RowG::NW], w1[RowG::NW];
                        load_col<FG, IQ, ST>(p0 + off, cs, w0);
                        load_col<FG, IQ, ST>(p0 + 16 + off, cs, w1);
                        accA.template add<FG>(bg, w0, w1, c0r, c0i, c1r, c1i);
                        load_col<FG, IQ, ST>(pB + off, cs, w0);
                        load_col<FG, IQ, ST>(pB + 16 + off, cs, w1);
                        accB.template add<FG>(bg, w0, w1, e0r, e0i, e1r, e1i);
                    }
                }
            }
        }
    }

#pragma unroll
    for (int b = 0; b < FB; ++b) {
        if (b0 + b < A.B) {
            float2 *x = reinterpret_cast<float2 *>(A.x) + (size_t)(b0 + b) * g.n_voxels + nA;
            if (validA) x[0] = make_float2(accA.re(b), accA.im(b));
            if (validB) x[1] = make_float2(accB.re(b), accB.im(b));
        }
    }
}

template <int FB, int ST>
cudaError_t launch_pair_t(const TileArgs &A, int n_chunks, cudaStream_t s) {
    const size_t smem = pair_smem_bytes(A.Q, A.w_tx != nullptr);
    auto kern = pair_kernel<FB, ST>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const long long blocks = (long long)((A.g.tiles_x + 1) / 2) * A.g.tiles_y * A.g.tiles_z;
    dim3 grid((unsigned)blocks, (unsigned)n_chunks);
    kern<<<grid, TILE_N, smem, s>>>(A);
    return cudaGetLastError();
}

}  // namespace das
