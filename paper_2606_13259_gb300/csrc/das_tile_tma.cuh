// das_tile_tma.cuh -- the voxel-tile kernel with TMA-staged sample windows.
//
// Same work and same arithmetic as tile_kernel (das_tile.cuh): one CTA per
// tile of 8 x 4 x 4 voxels and chunk of FB frames, one voxel per thread, FB
// accumulators in registers, no atomics.  The difference is how the two
// interpolation taps reach the registers.  For every (element, transmit) item
// the rows any voxel of the tile can need form one contiguous window of
// `umax` rows of z[chunk][q][m][.][FB]; thread 0 brings it into shared memory
// with a single bulk asynchronous copy (cp.async.bulk, completion counted on
// an mbarrier), up to TMA_STAGES items ahead of the consumers; a stage is
// refilled once each of the four warps has arrived on the stage's "empty"
// mbarrier, so warps drift apart by up to TMA_STAGES items instead of meeting
// at a CTA-wide barrier for every item.  Threads then read
// their two rows from shared memory, where lanes of a quarter-warp that need
// up to four different rows do not conflict, instead of from L1, where every
// distinct line costs a separate data-return wavefront.
//
// Window bound: with f = rf + t + delta the fractional delay of a voxel,
// |delta| <= a R (R the tile radius) and t >= tmin (per tile and transmit,
// from the prepare kernel), so floor(f) >= floor(rf + tmin - a R) and the
// span of floor(f) + 1 over the tile is at most 4 a R + 3 rows.  A voxel whose
// rows fall outside the window anyway reads them from global memory.
//
// Waits on the mbarriers are bounded by 1 s of wall time; on expiry the warp
// sets bit 0 of the plan's error word and a flag in shared memory on which the
// other warps' waits give up too, then the CTA waits (bounded) for the copies
// it has in flight and returns.
#pragma once

#include "das_async.cuh"
#include "das_tile.cuh"

namespace das {

constexpr int TMA_STAGES = 10;

// First row and row count of the staged window of one (element, transmit).
__device__ __forceinline__ void item_window(int tb, int rb, float rf, float tmin, float win_lo, int umax, int K,
                                            int &ks, int &cnt) {
    const int kw0 = tb + rb + (int)floorf(rf + tmin - win_lo);
    const int kend = min(kw0 + umax, K);
    ks = max(kw0, 0);
    cnt = max(kend - ks, 0);
}

// One (tile, frame chunk) of one plan; `smem` is the CTA's dynamic shared
// memory (tile_tma_smem_bytes).  Returns false when a bounded wait expired.
// Called by tile_tma_kernel (one launch per plan) and by the persistent
// batch kernel (many plans, one launch).
template <int FB, bool IQ, int ST, int MODE>
__device__ __forceinline__ bool tile_tma_body(const TileArgs &A, const long long tile, const int chunk,
                                              unsigned char *smem, const unsigned grid_x) {
    using Row = FrameRow<FB, IQ, ST>;
    constexpr int SZ = Row::SZ;
    constexpr int RB = FB * SZ;  // bytes per staged row
    static_assert(RB % 16 == 0, "staged rows must be whole 16-byte vectors");
    const int Q = A.Q;
    const int umax = A.umax;
    const bool has_w = A.w_tx != nullptr;
    unsigned char *stages = smem;                                                        // [S][umax][RB]
    uint64_t *mbar = reinterpret_cast<uint64_t *>(stages + (size_t)TMA_STAGES * umax * RB);  // [S] full
    uint64_t *ebar = mbar + TMA_STAGES;                                                  // [S] empty
    uint64_t *pbar = ebar + TMA_STAGES;                                                  // [2] test hook, pad
    int2 *s_win = reinterpret_cast<int2 *>(pbar + 2);                                   // [S] (first row, rows)
    float4 *s_eg = reinterpret_cast<float4 *>(s_win + TMA_STAGES + (TMA_STAGES & 1));  // [128]
    float4 *s_en = s_eg + TILE_N;                                                        // [128]
    float *s_t = reinterpret_cast<float *>(s_en + TILE_N);                              // [Q][128]
    float *s_w = s_t + Q * TILE_N;                                                       // [Q][128]
    float *s_tmin = s_w + (has_w ? Q * TILE_N : 0);                                      // [Q]
    int *s_erb = reinterpret_cast<int *>(s_tmin + Q);                                    // [128]
    int *s_em = s_erb + TILE_N;                                                          // [128]
    int *s_tb = s_em + TILE_N;                                                           // [Q]
    int *s_cnt = s_tb + Q;                                                               // [4]
    int *s_abort = s_cnt + 4;                                                            // [1]

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
    const unsigned char *zc = reinterpret_cast<const unsigned char *>(A.z) +
                              (size_t)chunk * Q * A.M * A.K * (size_t)RB;  // this chunk
    const size_t qstride = (size_t)A.M * A.K * RB;

    __syncthreads();  // a previous body call on this CTA is done with shared memory and barriers
    for (int q = 0; q < Q; ++q) {
        s_t[q * TILE_N + tid] = A.tx_t[(tile * Q + q) * TILE_N + tid];
        if (has_w) s_w[q * TILE_N + tid] = A.w_tx[(tile * Q + q) * TILE_N + tid];
    }
    for (int q = tid; q < Q; q += TILE_N) {
        s_tb[q] = A.tx_tb[tile * Q + q];
        s_tmin[q] = A.tx_tmin[tile * Q + q];
    }
    if (tid == 0) {
        for (int s = 0; s < TMA_STAGES; ++s) {
            mbar_init(&mbar[s], 1);               // completes when the copy has landed
            mbar_init(&ebar[s], TILE_N / 32);     // completes when every warp is done with the stage
        }
        mbar_init(pbar, 1);                       // nothing arrives on it (test hook)
        mbar_init_fence();
        *s_abort = 0;
    }

    FrameAcc<FB, IQ, ST> acc;
    acc.zero();

    // Thread 0 stages item i (element j = i / Q, transmit q = i % Q) of the
    // current element block into stage (g0 + i) % S, once every warp is done
    // with that stage's previous item.  Returns false if that wait expired.
    int n_issued = 0;  // thread 0: items of the current element block issued so far
    auto issue = [&](long long g0, int i) -> bool {
        const int j = i / Q, q = i - j * Q;
        const long long gi = g0 + i;
        if (gi >= TMA_STAGES &&
            !mbar_wait_ns(&ebar[gi % TMA_STAGES], (uint32_t)(((gi / TMA_STAGES) - 1) & 1), WAIT_NS, s_abort))
            return false;
        uint64_t *bar = &mbar[gi % TMA_STAGES];
        int ks, cnt;
        item_window(s_tb[q], s_erb[j], s_en[j].w, s_tmin[q], A.win_lo, umax, A.K, ks, cnt);
        s_win[gi % TMA_STAGES] = make_int2(ks, cnt);  // published to the consumers by the arrive below
        if (cnt > 0) {
            const uint32_t bytes = (uint32_t)cnt * RB;
            mbar_arrive_expect_tx(bar, bytes);
            bulk_copy_g2s(stages + (size_t)(gi % TMA_STAGES) * umax * RB,
                          zc + q * qstride + ((size_t)s_em[j] * A.K + ks) * RB, bytes, bar);
        } else {
            mbar_arrive(bar);
        }
        ++n_issued;
        return true;
    };

    const int lane = tid & 31, warp = tid >> 5;
    long long g0 = 0;  // items staged in earlier element blocks (mbarrier phase bookkeeping)
    bool aborted = false;
    for (int m0 = 0; m0 < A.M && !aborted; m0 += TILE_N) {
        __syncthreads();  // previous block's records and stages are no longer read
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

        const int n_items = total * Q;
        volatile int *abort_flag = s_abort;
        n_issued = 0;
        if (tid == 0)
            for (int i = 0; i < TMA_STAGES && i < n_items; ++i)
                if (!issue(g0, i)) { atomicOr(A.err, 1); *abort_flag = 1; break; }

        int j = 0, q = 0;
        bool inside = false;
        float r = 0.f;
        float4 G = make_float4(0.f, 0.f, 0.f, 0.f), Nn = G;
        int Rb = 0, mm = 0;
        for (int i = 0; i < n_items; ++i) {
            if (q == 0) {
                // (voxel, element) part of the geometry, once per element
                G = s_eg[j];
                Nn = s_en[j];
                Rb = s_erb[j];
                mm = s_em[j];
                const float ex = G.x + dx, ey = G.y + dy, ez = G.z + dz;
                inside = valid;
                if (A.thr >= 0.f) {
                    const float zax = fmaf(ex, Nn.x, fmaf(ey, Nn.y, ez * Nn.z));
                    const float cx = fmaf(ey, Nn.z, -ez * Nn.y), cy = fmaf(ez, Nn.x, -ex * Nn.z),
                                cz = fmaf(ex, Nn.y, -ey * Nn.x);
                    const float rho2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
                    inside = inside && (zax > 0.f) && (rho2 <= A.thr * zax * zax);
                }
                const float d = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
                const float num = fmaf(2.f, fmaf(G.x, dx, fmaf(G.y, dy, G.z * dz)), dd);
                r = Nn.w + A.a * __fdividef(num, d + G.w);
            }
            const long long gi = g0 + i;
            const int st = (int)(gi % TMA_STAGES);
            // warp-uniform decision: thread 0 may set the flag in its refill wait
            // while the other lanes of its warp are already past this point, so
            // the warp reconverges here and leaves together (a lane that left
            // alone would leave the others waiting at __syncwarp below)
            if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
            // test hook (das_plan_set_wait_test): warp 1 of the first CTA waits
            // on a barrier nothing arrives on for its first item, so it runs out
            const bool probe = A.probe && tile == 0 && chunk == 0 && gi == 0 && warp == 1;
            // (a warp that gives up because another one did takes the same exit)
            const bool timed_out = probe ? !mbar_wait_ns(pbar, 0u, A.wait_ns ? A.wait_ns : WAIT_NS)
                                         : !mbar_wait_ns(&mbar[st], (uint32_t)((gi / TMA_STAGES) & 1), WAIT_NS,
                                                         abort_flag);
            if (__any_sync(0xffffffffu, timed_out)) {
                if (lane == 0) atomicOr(A.err, 1);
                *abort_flag = 1;
                break;
            }
            const float f = r + s_t[q * TILE_N + tid];
            const float fl = floorf(f);
            const float al = f - fl;
            const int k = s_tb[q] + Rb + (int)fl;
            if (inside && (unsigned)k <= (unsigned)(A.K - 2)) {
                float w = has_w ? s_w[q * TILE_N + tid] : 1.f;
                if (ST != ST_F32) w *= __ldg(A.scale + (size_t)q * A.M + mm);
                float c0r, c0i = 0.f, c1r, c1i = 0.f;
                if constexpr (IQ) {
                    float sn, cs;
                    __sincosf(A.theta * (al - 0.5f), &sn, &cs);
                    const float uhr = cs * A.hr - sn * A.hi, uhi = cs * A.hi + sn * A.hr;
                    const float ubr = cs * A.hr + sn * A.hi, ubi = sn * A.hr - cs * A.hi;
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
                const int2 win = s_win[st];
                const int u = k - win.x;
                if (u >= 0 && u + 1 < win.y) {
                    // rows u and u+1 of the staged window, FG frames at a time
                    constexpr int FG = (FB % 4 == 0 && (4 * SZ) % 16 == 0) ? 4 : FB;
                    constexpr int GW = FG * SZ / 4;  // 32-bit words per group and row
                    static_assert((FG * SZ) % 16 == 0, "frame groups must be whole 16-byte vectors");
                    const uint32_t a0 = smem_addr(stages) + (uint32_t)((st * umax + u) * RB);
#pragma unroll
                    for (int bg = 0; bg < FB; bg += FG) {
                        uint32_t w0[GW], w1[GW];
#pragma unroll
                        for (int v = 0; v < GW / 4; ++v) {
                            const uint4 x0 = lds128(a0 + bg * SZ + 16 * v), x1 = lds128(a0 + RB + bg * SZ + 16 * v);
                            w0[4 * v] = x0.x; w0[4 * v + 1] = x0.y; w0[4 * v + 2] = x0.z; w0[4 * v + 3] = x0.w;
                            w1[4 * v] = x1.x; w1[4 * v + 1] = x1.y; w1[4 * v + 2] = x1.z; w1[4 * v + 3] = x1.w;
                        }
                        acc.template add<FG>(bg, w0, w1, c0r, c0i, c1r, c1i);
                    }
                } else {
                    uint32_t w0[Row::NW], w1[Row::NW];
                    const unsigned char *p0 = zc + q * qstride + ((size_t)mm * A.K + k) * RB;
                    Row::load(p0, w0);
                    Row::load(p0 + RB, w1);
                    acc.template add<FB>(0, w0, w1, c0r, c0i, c1r, c1i);
                }
            }
            // this warp is done with stage st
            __syncwarp();
            if (lane == 0) mbar_arrive(&ebar[st]);
            // refill the stage of the previous item (one item of slack for the other warps)
            if (tid == 0 && i >= 1 && i - 1 + TMA_STAGES < n_items && !*abort_flag)
                if (!issue(g0, i - 1 + TMA_STAGES)) { atomicOr(A.err, 1); *abort_flag = 1; }
            if (++q == Q) {
                q = 0;
                ++j;
            }
        }
        __syncthreads();
        if (*abort_flag) {
            aborted = true;
            if (tid == 0) {
                // copies that can still be in flight: the last S items issued (every
                // earlier one was waited for through its stage's empty barrier)
                for (int d = n_issued - 1; d >= 0 && d >= n_issued - TMA_STAGES; --d) {
                    const long long gd = g0 + d;
                    mbar_wait_ns(&mbar[gd % TMA_STAGES], (uint32_t)((gd / TMA_STAGES) & 1), WAIT_NS);
                }
            }
        }
        g0 += n_items;
    }
    if (aborted) return false;

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
        if (valid) {
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
        double *red = reinterpret_cast<double *>(s_eg);  // element records are no longer read
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < TILE_N / 32; ++w) s += red[w];
            A.partial[(size_t)chunk * grid_x + tile] = s;
        }
    }
    return true;
}

// Resident CTAs per SM asked of the compiler (register budget 65536 / (128 x v)).
template <int FB> struct TmaOcc { static constexpr int v = FB <= 8 ? 6 : FB <= 12 ? 5 : 4; };

template <int FB, bool IQ, int ST, int MODE>
__global__ void __launch_bounds__(TILE_N, TmaOcc<FB>::v) tile_tma_kernel(const TileArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    tile_tma_body<FB, IQ, ST, MODE>(A, blockIdx.x, blockIdx.y, smem, gridDim.x);
}

inline size_t tile_tma_smem_bytes(int Q, bool has_w, int umax, int rb) {
    return (size_t)TMA_STAGES * umax * rb + sizeof(uint64_t) * (2 * TMA_STAGES + 2) +
           sizeof(int2) * (TMA_STAGES + (TMA_STAGES & 1)) + sizeof(float4) * 2 * TILE_N +
           sizeof(float) * ((size_t)Q * TILE_N * (has_w ? 2 : 1) + Q) + sizeof(int) * (2 * TILE_N + Q + 5);
}

template <int FB, bool IQ, int ST, int MODE>
cudaError_t launch_tile_tma_t(const TileArgs &A, int n_chunks, cudaStream_t s) {
    constexpr int RB = FB * SampleSize<IQ, ST>::v;
    const size_t smem = tile_tma_smem_bytes(A.Q, A.w_tx != nullptr, A.umax, RB);
    auto kern = tile_tma_kernel<FB, IQ, ST, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)n_tiles(A.g), (unsigned)n_chunks);
    kern<<<grid, TILE_N, smem, s>>>(A);
    return cudaGetLastError();
}

// The staged kernel where its rows are whole 16-byte vectors, staging is on
// (umax > 0) and the window buffers fit comfortably in shared memory; else
// the tile kernel reading rows from global memory (256-bit loads on request
// where rows are whole 32-byte vectors).
template <int FB, bool IQ, int ST, int MODE>
cudaError_t launch_tile_best(const TileArgs &A, int n_chunks, cudaStream_t s) {
    constexpr int RB = FB * SampleSize<IQ, ST>::v;
    if constexpr (RB % 16 == 0) {
        if (A.umax > 0 && !A.col && tile_tma_smem_bytes(A.Q, A.w_tx != nullptr, A.umax, RB) <= 96 * 1024)
            return launch_tile_tma_t<FB, IQ, ST, MODE>(A, n_chunks, s);
    }
    if constexpr (MODE == MODE_FWD && IQ && RB % 32 == 0) {
        if (A.w256) return launch_tile_t<FB, IQ, ST, MODE, LD_W256>(A, n_chunks, s);
    }
    if constexpr (ColShape<FB, IQ, ST>::ok) {
        if (A.col) return launch_tile_t<FB, IQ, ST, MODE, LD_COL>(A, n_chunks, s);
    }
    if (A.col) return cudaErrorInvalidValue;  // the data were laid out for a column read
    return launch_tile_t<FB, IQ, ST, MODE, LD_ROW>(A, n_chunks, s);
}

}  // namespace das
