// das_adjoint.cu -- adjoint delay-and-sum (image -> channel data), the exact
// conjugate transpose of the forward map of Eq. 2 (Sec. 2).
//
// Each forward term reads two samples, w e^{i theta tau} ((1 - a) y[k] + a y[k+1]);
// its adjoint sends conj(w e^{i theta tau}) (1 - a) x_n to y[k] and
// conj(w e^{i theta tau}) a x_n to y[k+1].  The kernel is element-major: one
// CTA owns one band of `rows` samples of the channel rows (q, m) of one
// element m, for a chunk of transmits and frames.  It accumulates the band in
// shared memory while it visits every voxel tile that can see the element and
// whose delays can reach the band (the tile's transmit row span from the
// prepare kernel, widened by the receive offset bound), and writes the band
// once, in the public layout y[b][q][m][k].  Most bands of a long record hold
// no echo and are written as zeros at once; the others split an element's
// work into pieces of similar size, so the grid is many short, balanced CTAs.
// No global atomics; every output value is written by exactly one CTA, zeros
// included.
//
// Delays use the same split as the forward kernels (float64 reference to the
// tile centre, float32 offsets; see das_internal.cuh).
//
// A thread owns one line of 8 voxels along x in a tile (16 lines per tile,
// 32 tiles in flight per CTA).  For each transmit it walks the line keeping
// the contributions to two consecutive sample rows in registers; neighbours
// along x mostly fall on the same or the next row, so a row is added to shared
// memory (one atomic per value) only when the walk leaves it, instead of once
// per voxel.
#include "das_internal.cuh"

namespace das {

constexpr int ADJ_THREADS = 512;  // 32 tiles x 16 voxel lines in flight per CTA
// CTAs per SM asked of the compiler: two (64 registers, a few spilled words)
// ran the differentiation workload's adjoint in 23.4 ms, one (96-114
// registers, no spills, half the warps) in 36.4 ms.
#ifndef ADJ_MINB
#define ADJ_MINB 2
#endif

struct AdjTileRec {
    float gx, gy, gz, d0;  // tile centre minus element, and its norm
    float rf;              // fractional part of the reference delay
    int rb;                // integer part
    int tile;
    int inside;            // 1: every row the tile can reach lies in this CTA's band
};

template <bool IQ, int FB>
__global__ void __launch_bounds__(ADJ_THREADS, ADJ_MINB) adjoint_kernel(const AdjArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int C = IQ ? 2 : 1;
    const int m = blockIdx.x;
    const int band = blockIdx.y % A.n_bands;
    const int q0 = (blockIdx.y / A.n_bands) * A.qc;
    const int nq = min(A.qc, A.Q - q0);
    const int b0 = blockIdx.z * FB;
    const int K = A.K;
    const int L = A.rows;
    const int R0 = band * L, R1 = min(R0 + L, K);  // rows of this CTA
    float *acc = reinterpret_cast<float *>(smem);                             // [qc][L][FB][C]
    AdjTileRec *recs = reinterpret_cast<AdjTileRec *>(acc + (size_t)A.qc * L * FB * C);  // [2 ADJ_THREADS]
    int *s_cnt = reinterpret_cast<int *>(recs + 2 * ADJ_THREADS);             // [ADJ_THREADS / 32]

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < A.qc * L * FB * C; i += ADJ_THREADS) acc[i] = 0.f;

    const GridDesc &g = A.g;
    const double rx = A.elem_pos[3 * m], ry = A.elem_pos[3 * m + 1], rz = A.elem_pos[3 * m + 2];
    const float4 nn = A.elem_nrm[m];
    const long long ntiles = n_tiles(g);

    // Thread = (tile slot, line): slot tid / 16 takes every 32nd candidate
    // tile, line tid % 16 the voxels (x = 0..7, y = line % 4, z = line / 4).
    const int slot = tid >> 4;
    const int line = tid & 15;
    const int ly = line & 3, lz = line >> 2;
    const float dy = (float)(g.sy * (ly - 0.5 * (TILE_Y - 1)));
    const float dz = (float)(g.sz * (lz - 0.5 * (TILE_Z - 1)));

    // Candidate tiles are gathered over scan passes of ADJ_THREADS tiles into a
    // buffer of 2 ADJ_THREADS records and processed once at least ADJ_THREADS
    // are waiting (or the scan is over), so that every processing round gives
    // each of the 32 tile slots a dozen tiles or more to balance.
    int nbuf = 0;  // records waiting in the buffer (the same value in every thread)
    for (long long t0 = 0; t0 < ntiles; t0 += ADJ_THREADS) {
        __syncthreads();  // acc is zeroed; s_cnt of the previous pass is no longer read
        // conservative tests in float32 whether any voxel of the tile sees the
        // element and can reach this CTA's rows; then, for the tiles that
        // pass, the float64 reference delay of element m to the tile centre
        const long long t = t0 + tid;
        bool cand = false;
        AdjTileRec rec;
        if (t < ntiles) {
            const int tx = (int)(t % g.tiles_x);
            const int ty = (int)((t / g.tiles_x) % g.tiles_y);
            const int tz = (int)(t / ((long long)g.tiles_x * g.tiles_y));
            double cx, cy, cz;
            tile_centre(g, tx, ty, tz, cx, cy, cz);
            const double Gx = cx - rx, Gy = cy - ry, Gz = cz - rz;
            rec.gx = (float)Gx; rec.gy = (float)Gy; rec.gz = (float)Gz;
            const float d0f = sqrtf(rec.gx * rec.gx + rec.gy * rec.gy + rec.gz * rec.gz);
            cand = true;
            if (A.thr >= 0.f) {
                const float z0 = rec.gx * nn.x + rec.gy * nn.y + rec.gz * nn.z;
                const float ux = rec.gy * nn.z - rec.gz * nn.y, uy = rec.gz * nn.x - rec.gx * nn.z,
                            uz = rec.gx * nn.y - rec.gy * nn.x;
                const float rho0 = sqrtf(ux * ux + uy * uy + uz * uz);
                const float zmax = z0 + A.tile_radius;
                const float rmin = fmaxf(rho0 - A.tile_radius, 0.f);
                cand = (zmax > 0.f) && (rmin * rmin <= A.thr * zmax * zmax * 1.001f);
            }
            if (cand) {
                // rows k of the tile lie in tb + Rb + floor(rest + rf + offset) with
                // |offset| <= a R: [span.x + Rb - aRi, span.y + Rb + aRi]; taps reach k + 1
                const int rbf = (int)floorf(A.a * d0f);
                const int2 sp = __ldg(A.tx_span + t);
                const int klo = sp.x + rbf - A.aRi, khi = sp.y + rbf + A.aRi;
                cand = klo < R1 && khi + 1 >= R0;
                rec.inside = (klo >= R0 && khi + 1 < R1) ? 1 : 0;
            }
            if (cand) {
                const double D0 = sqrt(Gx * Gx + Gy * Gy + Gz * Gz);
                const double Rd = A.ad * D0;
                const double Rf = floor(Rd);
                rec.d0 = (float)D0;
                rec.rf = (float)(Rd - Rf);
                rec.rb = (int)Rf;
                rec.tile = (int)t;
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, cand);
        if (lane == 0) s_cnt[warp] = __popc(bal);
        __syncthreads();
        int off = 0, total = 0;
        for (int w = 0; w < ADJ_THREADS / 32; ++w) {
            const int c = s_cnt[w];
            off += (w < warp) ? c : 0;
            total += c;
        }
        if (cand) recs[nbuf + off + __popc(bal & ((1u << lane) - 1u))] = rec;
        nbuf += total;
        if (nbuf < ADJ_THREADS && t0 + ADJ_THREADS < ntiles) continue;  // gather more first
        __syncthreads();

        for (int c = slot; c < nbuf; c += ADJ_THREADS / 16) {
            const AdjTileRec R = recs[c];
            const int tile = R.tile;
            const int tx = tile % g.tiles_x;
            const int ty = (tile / g.tiles_x) % g.tiles_y;
            const int tz = tile / (g.tiles_x * g.tiles_y);
            const int iy = ty * TILE_Y + ly, iz = tz * TILE_Z + lz;
            if (iy >= g.ny || iz >= g.nz) continue;
            // receive geometry of the 8 voxels of the line (transmit independent)
            float r[TILE_X];
            unsigned live = 0u;  // bit x: voxel inside the grid and the aperture
#pragma unroll
            for (int x = 0; x < TILE_X; ++x) {
                const float dx = (float)(g.sx * (x - 0.5 * (TILE_X - 1)));
                const float ex = R.gx + dx, ey = R.gy + dy, ez = R.gz + dz;
                bool in = tx * TILE_X + x < g.nx;
                if (A.thr >= 0.f) {
                    const float zax = fmaf(ex, nn.x, fmaf(ey, nn.y, ez * nn.z));
                    const float ux = fmaf(ey, nn.z, -ez * nn.y), uy = fmaf(ez, nn.x, -ex * nn.z),
                                uz = fmaf(ex, nn.y, -ey * nn.x);
                    const float rho2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
                    in = in && (zax > 0.f) && (rho2 <= A.thr * zax * zax);
                }
                const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float d = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
                const float num = fmaf(2.f, fmaf(R.gx, dx, fmaf(R.gy, dy, R.gz * dz)), dd);
                r[x] = R.rf + A.a * __fdividef(num, d + R.d0);
                live |= (in ? 1u : 0u) << x;
            }
            if (live == 0u) continue;
            const long long nrow = ((long long)iz * g.ny + iy) * g.nx + (long long)tx * TILE_X;
            // with one frame per CTA the line's image values stay in registers across transmits
            constexpr bool HOIST = FB == 1;
            float xh[HOIST ? TILE_X * C : 1];
            if constexpr (HOIST) {
#pragma unroll
                for (int x = 0; x < TILE_X; ++x) {
                    float xr = 0.f, xi = 0.f;
                    if (((live >> x) & 1u) && b0 < A.B) {
                        const size_t o = (size_t)b0 * g.n_voxels + nrow + x;
                        if constexpr (IQ) {
                            const float2 v = __ldg(reinterpret_cast<const float2 *>(A.x) + o);
                            xr = v.x;
                            xi = v.y;
                        } else {
                            xr = __ldg(reinterpret_cast<const float *>(A.x) + o);
                        }
                    }
                    xh[x * C] = xr;
                    if constexpr (IQ) xh[x * C + 1] = xi;
                }
            }
            for (int qq = 0; qq < nq; ++qq) {
                const int q = q0 + qq;
                const size_t tq = (size_t)tile * A.Q + q;
                const int kb = __ldg(A.tx_tb + tq) + R.rb;
                // this transmit's rows of the tile against the band (not needed when
                // every row the tile can reach lies in the band)
                if (!R.inside && (kb + (int)floorf(__ldg(A.tx_tmin + tq)) - A.aRi >= R1 ||
                                  kb + (int)floorf(__ldg(A.tx_tmax + tq)) + A.aRi + 2 < R0))
                    continue;
                float *const arow = acc + (size_t)qq * L * FB * C;  // row k at arow + (k - R0) FB C
                // running rows kc and kc + 1 (kc = -4: none yet)
                int kc = -4;
                float a0[FB * C], a1[FB * C];
#pragma unroll
                for (int i = 0; i < FB * C; ++i) a0[i] = a1[i] = 0.f;
                // transmit rests of the line's 8 voxels: tile lanes vbase + 0..3 (x = 0..3)
                // and vbase + 8..11 (x = 4..7), two aligned 16-byte loads
                const int vbase = ((ly & 1) << 2) | (((ly >> 1) << 1) << 3) | (lz << 5);
                const float4 t03 = __ldg(reinterpret_cast<const float4 *>(A.tx_t + tq * TILE_N + vbase));
                const float4 t47 = __ldg(reinterpret_cast<const float4 *>(A.tx_t + tq * TILE_N + vbase + 8));
                const float tl[TILE_X] = {t03.x, t03.y, t03.z, t03.w, t47.x, t47.y, t47.z, t47.w};
#pragma unroll
                for (int x = 0; x < TILE_X; ++x) {
                    if (!((live >> x) & 1u)) continue;
                    // tile lane of voxel (x, ly, lz) (inverse of lane_offset)
                    const int vl = ((x & 3) | ((ly & 1) << 2)) | (((x >> 2) | ((ly >> 1) << 1)) << 3) | (lz << 5);
                    const float f = r[x] + tl[x];
                    const float fl = floorf(f);
                    const float al = f - fl;
                    const int k = kb + (int)fl;
                    if ((unsigned)k > (unsigned)(K - 2)) continue;
                    if (k + 1 < R0 || k >= R1) continue;  // both taps outside the band
                    const float w = A.w_tx ? __ldg(A.w_tx + tq * TILE_N + vl) : 1.f;
                    float c0r, c0i = 0.f, c1r, c1i = 0.f;
                    if constexpr (IQ) {
                        float sn, cs;
                        // e^{i th a} directly, e^{-i th (1-a)} = e^{i th a} e^{-i th}
                        __sincosf(A.theta * al, &sn, &cs);
                        const float uhr = cs, uhi = sn;
                        const float ubr = cs * A.er - sn * A.ei, ubi = cs * A.ei + sn * A.er;
                        const float w0 = w * (1.f - al), w1 = w * al;
                        // conjugated coefficients of the two taps (pre-rotated sample domain)
                        c0r = w0 * uhr; c0i = -w0 * uhi; c1r = w1 * ubr; c1i = -w1 * ubi;
                    } else {
                        c0r = w * (1.f - al);
                        c1r = w * al;
                    }
                    // rows kc, kc + 1 that the new pair (k, k + 1) no longer covers go to
                    // shared memory (those of the band; the rest belong to other CTAs)
                    const bool keep0 = kc == k || kc == k + 1;
                    const bool keep1 = kc + 1 == k || kc + 1 == k + 1;
                    if (kc >= R0 && kc < R1 && !keep0) {
                        float *p = arow + (size_t)(kc - R0) * FB * C;
#pragma unroll
                        for (int i = 0; i < FB * C; ++i) atomicAdd(p + i, a0[i]);
                    }
                    if (kc + 1 >= R0 && kc + 1 < R1 && !keep1) {
                        float *p = arow + (size_t)(kc + 1 - R0) * FB * C;
#pragma unroll
                        for (int i = 0; i < FB * C; ++i) atomicAdd(p + i, a1[i]);
                    }
                    // carry what stays into the new pair's slots
                    float n0[FB * C], n1[FB * C];
#pragma unroll
                    for (int i = 0; i < FB * C; ++i) {
                        n0[i] = kc == k ? a0[i] : (kc + 1 == k ? a1[i] : 0.f);
                        n1[i] = kc == k + 1 ? a0[i] : (kc == k ? a1[i] : 0.f);
                    }
                    kc = k;
#pragma unroll
                    for (int b = 0; b < FB; ++b) {
                        float xr = 0.f, xi = 0.f;
                        if constexpr (HOIST) {
                            xr = xh[x * C];
                            if constexpr (IQ) xi = xh[x * C + 1];
                        } else if (b0 + b < A.B) {
                            const size_t o = (size_t)(b0 + b) * g.n_voxels + nrow + x;
                            if constexpr (IQ) {
                                const float2 v = __ldg(reinterpret_cast<const float2 *>(A.x) + o);
                                xr = v.x;
                                xi = v.y;
                            } else {
                                xr = __ldg(reinterpret_cast<const float *>(A.x) + o);
                            }
                        }
                        if constexpr (IQ) {
                            a0[2 * b] = n0[2 * b] + (c0r * xr - c0i * xi);
                            a0[2 * b + 1] = n0[2 * b + 1] + (c0r * xi + c0i * xr);
                            a1[2 * b] = n1[2 * b] + (c1r * xr - c1i * xi);
                            a1[2 * b + 1] = n1[2 * b + 1] + (c1r * xi + c1i * xr);
                        } else {
                            a0[b] = n0[b] + c0r * xr;
                            a1[b] = n1[b] + c1r * xr;
                        }
                    }
                }
                if (kc >= R0 && kc < R1) {
                    float *p = arow + (size_t)(kc - R0) * FB * C;
#pragma unroll
                    for (int i = 0; i < FB * C; ++i) atomicAdd(p + i, a0[i]);
                }
                if (kc + 1 >= R0 && kc + 1 < R1) {
                    float *p = arow + (size_t)(kc + 1 - R0) * FB * C;
#pragma unroll
                    for (int i = 0; i < FB * C; ++i) atomicAdd(p + i, a1[i]);
                }
            }
        }
        __syncthreads();  // the buffered records are processed
        nbuf = 0;
    }
    __syncthreads();

    // Write the owned rows in the public layout; IQ rows leave the pre-rotated
    // domain through conj(e^{i theta k}).
    for (int qq = 0; qq < nq; ++qq) {
        const int q = q0 + qq;
        for (int b = 0; b < FB; ++b) {
            if (b0 + b >= A.B) break;
            const size_t row = (((size_t)(b0 + b) * A.Q + q) * A.M + m) * (size_t)K;
            for (int k = R0 + tid; k < R1; k += ADJ_THREADS) {
                const float *a = acc + ((size_t)qq * L + (k - R0)) * FB * C + b * C;
                if constexpr (IQ) {
                    const float2 rt = A.rot ? A.rot[k] : make_float2(1.f, 0.f);
                    reinterpret_cast<float2 *>(A.y)[row + k] =
                        make_float2(a[0] * rt.x + a[1] * rt.y, a[1] * rt.x - a[0] * rt.y);
                } else {
                    reinterpret_cast<float *>(A.y)[row + k] = a[0];
                }
            }
        }
    }
}

size_t adjoint_smem_bytes(int qc, int rows, int fb, int iq) {
    return sizeof(float) * (size_t)qc * rows * fb * (iq ? 2 : 1) + sizeof(AdjTileRec) * 2 * ADJ_THREADS +
           sizeof(int) * (ADJ_THREADS / 32);
}

template <bool IQ, int FB>
static cudaError_t launch_adj_t(const AdjArgs &A, cudaStream_t s) {
    const size_t smem = adjoint_smem_bytes(A.qc, A.rows, FB, IQ);
    auto kern = adjoint_kernel<IQ, FB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long gy = (long long)((A.Q + A.qc - 1) / A.qc) * A.n_bands;
    if (gy > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)A.M, (unsigned)gy, (unsigned)((A.B + FB - 1) / FB));
    kern<<<grid, ADJ_THREADS, smem, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const AdjArgs &A, int iq, cudaStream_t s) {
    switch (A.fb) {
    case 1: return iq ? launch_adj_t<true, 1>(A, s) : launch_adj_t<false, 1>(A, s);
    case 2: return iq ? launch_adj_t<true, 2>(A, s) : launch_adj_t<false, 2>(A, s);
    case 4: return iq ? launch_adj_t<true, 4>(A, s) : launch_adj_t<false, 4>(A, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace das
