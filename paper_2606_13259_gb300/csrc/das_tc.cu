// das_tc.cu -- forward DAS of IQ data as a tensor-core contraction on
// sm_103a: tcgen05.mma with the weights and the accumulator in tensor memory
// (TMEM) and the sample windows brought into shared memory by TMA.
//
// Formulation (the tile reformulation of the paper's tensor-core kernel,
// Sec. 3.4, Alg. 3, regrouped for the 128-row MMA of this GPU).  For a tile
// of 128 voxels (one MMA row each), one chunk of bc frames and one
// (element m, transmit q) item, the part of Eq. 2 contributed by the item is
//
//     X[v][b] += sum_u W[v][u] Z[k0 + u][b],      u = 0 .. U-1  (U = 16 rows),
//
// where Z are the pre-rotated samples (z[k] = y[k] e^{i theta k}) of the
// item's window of rows k0 .. k0 + U - 1, and row v of W holds the two
// interpolation weights of voxel v, (1 - alpha) e^{i theta alpha} at
// u = k - k0 and alpha e^{-i theta (1 - alpha)} at u + 1, times the
// apodisation; every other entry is zero.  In real arithmetic, with
// W = Wr + i Wi and Z = Zr + i Zi,
//
//     [Xr | Xi] += [Wr | Wi] . [[Zr, Zi], [-Zi, Zr]],
//
// one MMA of M = 128, N = 2 bc (padded to a multiple of 16, at most 256) and
// K = 2 U = 32 (two K = 16 steps of kind::f16), accumulated in float32 in
// TMEM.  The tensor core's float32 accumulation loses a little of the running
// sum at every step (measured as a gain deficit that grows in proportion to
// the number of steps), so the items of a tile are summed in chains of a
// bounded number of sub-items: at the end of a chain the builder threads add
// D into the image with ordinary float32 arithmetic and the next chain starts
// from zero.
//
// Window of an item.  With f = rf + t + delta (das_internal.cuh), t between
// the tile's smallest and largest transmit rest (prepare kernel) and delta =
// a (|G + D| - |G|) bounded below by the tangent plane, a u.D >= -a sum_i
// |u_i| h_i, and above by min(a u.D + a R^2 / (2 |G|), a R) (G the element to
// tile-centre vector, u = G / |G|, h the half extents of the tile, R its
// radius), every k of the tile lies in [klo, khi] computed from per-item
// values alone.  Each thread derives the same [klo, khi], so the producer can
// fetch windows ahead of the threads that build W.  Items whose range spans
// more than U - 1 = 15 values of k are split into several MMA sub-items with
// windows 15 rows apart (none at the workloads of the paper).
//
// Operand layouts.
//   A (W): TMEM, lanes = voxels (tile lane order), 16 columns of 32 bits per
//          stage = 32 16-bit values, K-major: columns 0-7 Wr (u = 0..15),
//          8-15 Wi.  A ring of sa stages (2 .. 16).
//   B (window): shared memory, MN-major without swizzle.  The relayout
//          stores the channel data as z[c][q m][n / 8][plane][k][8] 16-bit
//          values, plane 0 = [Zr | Zi] and plane 1 = [-Zi | Zr] along n, so
//          one 4-D TMA box (16 rows x 8 values, 2, n / 8, 1) at element
//          8 k0 lands as core matrices of 8 n x 8 K values (128 B):
//          K-direction stride 128 B, n-direction stride 512 B.  Rows outside
//          0 .. K-1 arrive as zeros.
//   D: TMEM columns 0 .. n-1, lanes = voxels.
//
// CTA roles (G 128-thread builder groups + 2 warps): the builder threads
// compute the work list and build W (thread = voxel = TMEM lane) and store D;
// lanes of the next warp issue the window copies; lane 0 of the last warp
// issues the MMAs and their commits.  The roles hand sub-items over in
// bundles of H (two where the tensor memory holds two bundles of W stages):
// group g builds the bundles with index = g mod G.  Each hand-off of the
// MMA-issuing thread (a barrier test, a commit) costs it about as much as an
// MMA, and that thread's serial work, not the tensor core, bounds the kernel,
// so a bundle takes one test of each full barrier and one commit for H
// sub-items.  Barriers: fullA (one arrival per builder warp of the group),
// fullB (TMA transaction bytes of the bundle's windows), empty
// (tcgen05.commit of the bundle's MMAs: it frees the bundle's window slots
// and W stages alike), accFull (commit after the last MMA of a chain).
// Every wait is bounded; on expiry the CTA sets bit 2 of the plan's error
// word, drains what it has in flight and leaves without writing its image
// tile.
#include "das_async.cuh"
#include "das_tc.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

namespace das {

// A CTA has G groups of four builder warps (G = 2 with two CTAs per SM, 4 with
// one), one producer warp and one MMA warp.
__host__ __device__ constexpr int tc_threads(int G) { return G * TILE_N + 64; }
constexpr int TC_U = 16;        // window rows per sub-item
constexpr int TC_KV = TC_U - 1; // values of k a sub-item covers
constexpr int TC_MAX_SA = 16;   // W stages in TMEM (set per launch)

constexpr int TC_ACOLS = 16;    // TMEM columns per W stage
constexpr int TC_LIST_MAX = 4096;    // sub-items per list round (largest list)
constexpr int TC_MAX_SB = 24;
constexpr int TC_PRODUCERS = 4;  // producer lanes issuing window copies
constexpr float TC_MARGIN = 0.02f;  // samples

// ---------------------------------------------------------------------------
// tcgen05 / TMA primitives (inline PTX)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// D[tmem] (+)= A[tmem] . B[smem], kind::f16, one CTA.
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once every MMA this thread issued so far has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

// Shared-memory matrix descriptor, no swizzle: start address, K-direction and
// MN-direction strides between 8 x 16-byte core matrices (bytes).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t k_stride, uint32_t mn_stride) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((k_stride >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((mn_stride >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: float32 accumulator, A and B both f16
// (or both bf16), A K-major, B MN-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t tc_idesc(int n, bool bf16) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | (1u << 16) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    if constexpr (BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

constexpr uint64_t TC_WAIT_NS = 1000000000ull;  // 1 s
#ifndef TC_SLEEP_HINT_NS
#define TC_SLEEP_HINT_NS 8192
#endif
constexpr uint32_t TC_SLEEP_NS = TC_SLEEP_HINT_NS;  // suspend-time hint of a waiting thread (0: none)

// One test of a barrier phase with the suspend-time hint.
__device__ __forceinline__ bool tc_try(uint64_t *bar, uint32_t parity) {
    return TC_SLEEP_NS != 0 ? mbar_try_wait_sleep(bar, parity, TC_SLEEP_NS) : mbar_try_wait(bar, parity);
}

// Wait limit of the pipeline's hand-offs: the plan's test setting, else 1 s.
__device__ __forceinline__ uint64_t tc_limit(const TcArgs &A) { return A.wait_ns ? A.wait_ns : TC_WAIT_NS; }

// Bounded wait (`limit` ns of wall time); gives up early when another role of
// the CTA, or another CTA, has recorded a timeout.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, volatile uint32_t *abort_flag, int *err,
                                        uint64_t limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1;; ++i) {
        if (tc_try(bar, parity)) return true;
        if ((i & 7u) == 0u) {
            if (*abort_flag || (*(volatile int *)err & 4)) {
                *abort_flag = 1u;
                return false;
            }
            if (global_ns() - t0 > limit) break;
        }
    }
    atomicOr(err, 4);
    *abort_flag = 1u;
    return false;
}

// mbarrier arrive by the threads whose predicate is set (no branch).
__device__ __forceinline__ void mbar_arrive_if(uint64_t *bar, bool p) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
        "@q mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n\t}" ::"r"(smem_addr(bar)),
        "r"((uint32_t)p)
        : "memory");
}

// Slow path of a whole warp's wait (the first try failed): every lane takes
// the same decisions, so the warp stays converged.
__device__ __noinline__ bool tc_wait_warp(uint64_t *bar, uint32_t parity, volatile uint32_t *abort_flag, int *err,
                                          uint64_t limit) {
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1;; ++i) {
        if (__all_sync(0xffffffffu, tc_try(bar, parity))) return true;
        if ((i & 7u) == 0u) {
            const bool give_up = __any_sync(0xffffffffu, *abort_flag != 0u || (*(volatile int *)err & 4) != 0 ||
                                                             global_ns() - t0 > limit);
            if (give_up) break;
        }
    }
    if ((threadIdx.x & 31) == 0) {
        if (!(*(volatile int *)err & 4) && !*abort_flag) atomicOr(err, 4);
        *abort_flag = 1u;
    }
    __syncwarp();
    return false;
}

// Sub-items of one item: the range [klo, khi] every k of the tile lies in,
// clipped to the valid rows; returns the number of 15-value windows (0: no
// term of the item can be valid).
__device__ __forceinline__ int tc_item(int tb, int rb, float rf, float tmin, float tmax, float2 gb, int K, int &klo) {
    int lo = tb + rb + (int)floorf(rf + tmin + gb.x);
    int hi = tb + rb + (int)floorf(rf + tmax + gb.y);
    lo = max(lo, 0);
    hi = min(hi, K - 2);
    klo = lo;
    return hi < lo ? 0 : (hi - lo) / TC_KV + 1;
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------

struct TcSmem {
    size_t bars, misc, sel, list, lw, eg, en, gb, erb, em, t, w, tb, tmin, tmax, total;
};

// Rows of the byte-permute selectors that place a W row's two values: for a
// window offset u (0 .. TC_KV - 1) and word c of a 16-value plane, the bytes of
// the 32-bit word (value u, value u + 1) that word c takes (0x44: zero
// bytes).  Row TC_KV: all words zero (an inactive voxel).
constexpr int TC_SEL_ROWS = TC_KV + 1;
__host__ __device__ inline uint32_t tc_sel(int u, int c) {
    if (u >= TC_KV) return 0x4444u;
    if (c == (u >> 1)) return (u & 1) ? 0x1044u : 0x3210u;  // (u, u+1) in word c, or u in its upper half
    if ((u & 1) && c == (u >> 1) + 1) return 0x4432u;      // u + 1 in the lower half of the next word
    return 0x4444u;
}

// Shared memory of one CTA: sb window stages, barriers, the element records
// of one block of eb elements and a sub-item list of list_cap entries.
__host__ __device__ inline TcSmem tc_smem_layout(int sb, int n, int Q, bool has_w, int eb, int list_cap) {
    TcSmem L{};
    size_t o = (size_t)sb * 64 * n;  // window stages (1024-aligned base)
    L.bars = o; o += 128 * 8;
    L.misc = o; o += 128 * 4;
    L.sel = o; o += (size_t)TC_SEL_ROWS * 8 * 4;
    L.list = o; o += (size_t)list_cap * 8;
    L.lw = o; o += (size_t)list_cap * 4;
    L.eg = o; o += (size_t)eb * 16;
    L.en = o; o += (size_t)eb * 16;
    L.gb = o; o += (size_t)eb * 8;
    L.erb = o; o += (size_t)eb * 4;
    L.em = o; o += (size_t)eb * 4;
    L.t = o; o += (size_t)Q * TILE_N * 4;
    L.w = o; o += has_w ? (size_t)Q * TILE_N * 4 : 0;
    L.tb = o; o += (size_t)Q * 4;
    L.tmin = o; o += (size_t)Q * 4;
    L.tmax = o; o += (size_t)Q * 4;
    L.total = o + 1024;  // alignment slack of the dynamic base
    return L;
}

// misc words of the kernel's shared memory
enum : int { MW_TMEM = 0, MW_ABORT = 1, MW_ISSUED = 2, MW_NEL = 3, MW_NLIST = 4, MW_NEXT = 5, MW_CNT = 8,
             MW_SCAN = 40 };  // MW_CNT, MW_SCAN: one word per builder warp (up to 32)

// D of a finished accumulation chain -> image, by the builder threads (whole
// warps).  Waits for the chain's MMAs (accFull phase `parity`; bounded by time
// only, since MMAs in flight must land before tensor memory is read or
// reused), then each thread moves its voxel's frames b_first, b_first + 1, ...
// in 16-frame blocks b_step apart: x = D smax, or x += D smax when x already
// holds the earlier chains (add).  read_d false: no MMA ran, the frames get D = 0.
__device__ __noinline__ void tc_store_d(const TcArgs &A, uint32_t taddr, uint64_t *accFull, uint32_t parity, bool add,
                                        bool read_d, volatile uint32_t *s_abort, int lane, int b_first, int b_step,
                                        int chunk, bool valid, long long nvox) {
    bool ok = true;
    if (read_d && lane == 0) {
        const uint64_t t0 = global_ns();
        while (!(ok = tc_try(accFull, parity)))
            if (global_ns() - t0 > TC_WAIT_NS) break;
        if (!ok) {
            atomicOr(A.err, 4);
            *s_abort = 1u;
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0) != 0 && *s_abort == 0u;
    __syncwarp();
    tc_fence_after();
    const float sm = *A.smax;
    for (int b0 = b_first; b0 < A.bc; b0 += b_step) {
        uint32_t re[16], im[16];
        if (read_d) {
            tmem_ld16(taddr + (uint32_t)b0, re);
            tmem_ld16(taddr + (uint32_t)(A.bc + b0), im);
            tmem_ld_wait();
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) re[i] = im[i] = 0u;
        }
        if (ok && valid) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int b = b0 + i;
                const long long frame = (long long)chunk * A.bc + b;
                if (b < A.bc && frame < A.B) {
                    float2 *px = A.x + frame * A.g.n_voxels + nvox;
                    float2 v = make_float2(__uint_as_float(re[i]) * sm, __uint_as_float(im[i]) * sm);
                    if (add) {
                        const float2 o = *px;
                        v = make_float2(o.x + v.x, o.y + v.y);
                    }
                    *px = v;
                }
            }
        }
    }
    tc_fence_before();
}

template <bool BF16, int G, int MINB, bool CHAIN, int HAND>
__global__ void __launch_bounds__(tc_threads(G), MINB) tc_kernel(const __grid_constant__ CUtensorMap zmap,
                                                                 const __grid_constant__ TcArgs A) {
    constexpr int NB = G * TILE_N;  // builder threads
    constexpr int EB = NB;          // element records per block (one element per builder thread)
    const int list_cap = A.list_cap;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    const int Q = A.Q, M = A.M, K = A.K, n = A.n, sb = A.sb;
    // sub-items per hand-off (a bundle), W bundle stages in tensor memory,
    // window bundle slots in shared memory, producer lanes
    constexpr uint32_t H = HAND;
    const uint32_t pa_n = (uint32_t)A.sa / H;
    const uint32_t pb_n = (uint32_t)A.sb / H, nprod = TC_PRODUCERS / H;
    const bool has_w = A.w_tx != nullptr;
    const TcSmem L = tc_smem_layout(sb, n, Q, has_w, EB, list_cap);
    const uint32_t stage_bytes = 64u * (uint32_t)n;
    unsigned char *sB = smem;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    // fullB / emptyB: one per window bundle slot; fullA / emptyA: one per W bundle stage
    uint64_t *fullB = bars, *emptyB = bars + TC_MAX_SB, *fullA = bars + 2 * TC_MAX_SB, *emptyA = fullA + TC_MAX_SA;
    uint64_t *accFull = emptyA + TC_MAX_SA;
    uint64_t *probe = accFull + 1;  // test hook: a barrier nothing arrives on
    uint32_t *misc = reinterpret_cast<uint32_t *>(smem + L.misc);
    volatile uint32_t *s_abort = misc + MW_ABORT;
    int2 *s_list = reinterpret_cast<int2 *>(smem + L.list);  // (window row, j | q << 9)
    float *s_lw = reinterpret_cast<float *>(smem + L.lw);     // storage scale ratio of the item
    float4 *s_eg = reinterpret_cast<float4 *>(smem + L.eg);
    float4 *s_en = reinterpret_cast<float4 *>(smem + L.en);
    float2 *s_gb = reinterpret_cast<float2 *>(smem + L.gb);
    int *s_erb = reinterpret_cast<int *>(smem + L.erb);
    int *s_em = reinterpret_cast<int *>(smem + L.em);
    float *s_t = reinterpret_cast<float *>(smem + L.t);
    float *s_w = reinterpret_cast<float *>(smem + L.w);
    int *s_tb = reinterpret_cast<int *>(smem + L.tb);
    float *s_tmin = reinterpret_cast<float *>(smem + L.tmin);
    float *s_tmax = reinterpret_cast<float *>(smem + L.tmax);
    uint32_t *s_sel = reinterpret_cast<uint32_t *>(smem + L.sel);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int vl = tid & (TILE_N - 1);  // voxel lane = TMEM lane of a builder thread
    const long long tile = blockIdx.x;
    const int chunk = blockIdx.y;
    const GridDesc &g = A.g;
    const int tx = (int)(tile % g.tiles_x);
    const int ty = (int)((tile / g.tiles_x) % g.tiles_y);
    const int tz = (int)(tile / ((long long)g.tiles_x * g.tiles_y));

    if (tid == 0) {
        for (uint32_t s = 0; s < pb_n; ++s) {
            mbar_init(&fullB[s], 1);
            mbar_init(&emptyB[s], 1);
        }
        for (uint32_t s = 0; s < pa_n; ++s) {
            mbar_init(&fullA[s], TILE_N / 32);  // one arrival per builder warp of the bundle's group
            mbar_init(&emptyA[s], 1);
        }
        mbar_init(accFull, 1);
        mbar_init(probe, 1);
        misc[MW_ABORT] = (*(volatile int *)A.err & 4) ? 1u : 0u;  // another CTA gave up: leave at once
        misc[MW_ISSUED] = 0u;
        mbar_init_fence();
    }
    if (warp == 0) {
        tmem_alloc(&misc[MW_TMEM], (uint32_t)A.ncols);
        tmem_relinquish();
    }
    if (tid < TILE_N) {
        for (int q = 0; q < Q; ++q) {
            s_t[q * TILE_N + tid] = A.tx_t[(tile * Q + q) * TILE_N + tid];
            if (has_w) s_w[q * TILE_N + tid] = A.w_tx[(tile * Q + q) * TILE_N + tid];
        }
    }
    for (int i = tid; i < TC_SEL_ROWS * 8; i += tc_threads(G)) s_sel[i] = tc_sel(i >> 3, i & 7);
    for (int q = tid; q < Q; q += tc_threads(G)) {
        s_tb[q] = A.tx_tb[tile * Q + q];
        s_tmin[q] = A.tx_tmin[tile * Q + q];
        s_tmax[q] = A.tx_tmax[tile * Q + q];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = misc[MW_TMEM];

    // voxel of a builder thread (both groups cover the same 128 voxels)
    int lx = 0, ly = 0, lz = 0;
    lane_offset(vl, lx, ly, lz);
    const int ix = tx * TILE_X + lx, iy = ty * TILE_Y + ly, iz = tz * TILE_Z + lz;
    const bool valid = tid < NB && ix < g.nx && iy < g.ny && iz < g.nz;
    double p0x, p0y, p0z;
    tile_centre(g, tx, ty, tz, p0x, p0y, p0z);
    const float dx = (float)(g.sx * (lx - 0.5 * (TILE_X - 1)));
    const float dy = (float)(g.sy * (ly - 0.5 * (TILE_Y - 1)));
    const float dz = (float)(g.sz * (lz - 0.5 * (TILE_Z - 1)));
    const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));

    // image rows of a builder thread: its voxel, its TMEM lane, its first 16-frame block
    const long long nvox = ((long long)iz * g.ny + iy) * g.nx + ix;
    const uint32_t lane_d = (uint32_t)((warp & 3) * 32) << 16;
    const int b_first = 16 * (tid >> 7);

    uint32_t base = 0;  // sub-items of earlier rounds (same value in every thread)
    // accumulation chains (same values in every thread): first sub-item of the
    // current chain, commits to accFull so far, whether x already holds a sum
    uint32_t chain0 = 0, n_commit = 0;
    bool folded = false;
    const size_t qm_base = (size_t)chunk * Q * M;
    bool stop = misc[MW_ABORT] != 0u;
    uint32_t tma_issued = 0;  // producer: window copies issued
    // position in the window ring of this thread's role (producer, MMA
    // issuer): slot, completed passes over the ring (its low bit is the phase)
    uint32_t b_slot = (warp == NB / 32 && (uint32_t)lane < nprod) ? (uint32_t)lane : 0u, b_pass = 0;
    uint32_t bbase = 0;  // bundles of earlier rounds (same value in every thread)
    // builders: W bundle stage of the group's next bundle (its bundles are grp,
    // grp + G, ... across rounds) and the uses of that stage before it; MMA
    // issuer: the same for its next bundle
    uint32_t bps = (uint32_t)(tid >> 7) % pa_n, bpass = (uint32_t)(tid >> 7) / pa_n;
    uint32_t mps = 0, mpass = 0;

    for (int m0 = 0; m0 < M; m0 += EB) {
        const int mend = min(M, m0 + EB);
        // ---- compaction of the candidate elements of this block (builder threads) ----
        {
            bool cand = false;
            float4 eg = make_float4(0.f, 0.f, 0.f, 0.f), en = eg;
            float2 gbv = make_float2(0.f, 0.f);
            int rb = 0;
            const int m = m0 + tid;
            if (tid < EB && m < mend) {
                const double rx = A.elem_pos[3 * m], ry = A.elem_pos[3 * m + 1], rz = A.elem_pos[3 * m + 2];
                const double Gx = p0x - rx, Gy = p0y - ry, Gz = p0z - rz;
                const double D0 = sqrt(Gx * Gx + Gy * Gy + Gz * Gz);
                const double R0 = A.ad * D0;
                const double Rf = floor(R0);
                rb = (int)Rf;
                const float4 nn = A.elem_nrm[m];
                eg = make_float4((float)Gx, (float)Gy, (float)Gz, (float)D0);
                en = make_float4(nn.x, nn.y, nn.z, (float)(R0 - Rf));
                if (eg.w > 1e-12f) {
                    // window bound offsets in float32 (0.02-sample margin); the
                    // reference delay above stays float64
                    const float inv = 1.f / eg.w;
                    const float lin = (fabsf(eg.x) * A.ahx + fabsf(eg.y) * A.ahy + fabsf(eg.z) * A.ahz) * inv;
                    const float curv = A.aR2h * inv;
                    gbv = make_float2(-lin - TC_MARGIN, fminf(lin + curv, A.aR) + TC_MARGIN);
                } else {
                    gbv = make_float2(-A.aR - TC_MARGIN, A.aR + TC_MARGIN);
                }
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
            if (tid < EB && lane == 0) misc[MW_CNT + warp] = __popc(bal);
            __syncthreads();
            if (tid < EB && cand) {
                int off = 0;
                for (int w = 0; w < warp; ++w) off += (int)misc[MW_CNT + w];
                const int idx = off + __popc(bal & ((1u << lane) - 1u));
                s_eg[idx] = eg;
                s_en[idx] = en;
                s_gb[idx] = gbv;
                s_erb[idx] = rb;
                s_em[idx] = m;
            }
            if (tid == 0) {
                int tot = 0;
                for (int w = 0; w < EB / 32; ++w) tot += (int)misc[MW_CNT + w];
                misc[MW_NEL] = (uint32_t)tot;
            }
            __syncthreads();
        }
        const int n_el = (int)misc[MW_NEL];
        const int P = n_el * Q;  // (element, transmit) pairs, element-major

        for (int p0 = 0; p0 < P;) {
            // A chain that has reached its length ends here: its MMAs are
            // committed now and the builders add D into the image once they
            // have built this round's list, so that the last MMAs finish
            // while the list is built (all threads take the same decision).
            const uint32_t issued = CHAIN ? misc[MW_ISSUED] : 0u;  // written before the last barrier
            const bool new_chain = CHAIN && base - chain0 >= (uint32_t)A.chain;
            const bool fold = new_chain && issued > chain0;
            if (fold && warp == NB / 32 + 1 && lane == 0) mma_commit(accFull);

            // ---- sub-item list of pairs p0 .. (as many as fit), by the builder threads ----
            const int per = (P - p0 + NB - 1) / NB;
            const int pa = min(P, p0 + tid * per), pe = min(P, pa + per);
            int cnt = 0;
            if (tid < NB) {
                for (int p = pa; p < pe; ++p) {
                    const int j = p / Q, q = p - j * Q;
                    int klo;
                    cnt += tc_item(s_tb[q], s_erb[j], s_en[j].w, s_tmin[q], s_tmax[q], s_gb[j], K, klo);
                }
            }
            // exclusive scan of cnt over the builder threads
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (tid < NB && lane == 31) misc[MW_SCAN + warp] = (uint32_t)incl;
            if (tid == 0) {
                misc[MW_NEXT] = (uint32_t)P;
                misc[MW_NLIST] = 0u;
            }
            __syncthreads();
            int off = incl - cnt;
            for (int w = 0; w < warp && w < NB / 32; ++w) off += (int)misc[MW_SCAN + w];
            if (tid < NB) {
                for (int p = pa; p < pe; ++p) {
                    const int j = p / Q, q = p - j * Q;
                    int klo;
                    int ns = tc_item(s_tb[q], s_erb[j], s_en[j].w, s_tmin[q], s_tmax[q], s_gb[j], K, klo);
                    if (off + ns > list_cap) {
                        if (ns > list_cap) {  // one pair wider than the whole list: keep what fits, flag it
                            if (off == 0) {
                                atomicOr(A.err, 8);
                                ns = list_cap;
                            }
                        }
                        if (off + ns > list_cap) {
                            atomicMin(&misc[MW_NEXT], (uint32_t)p);
                            break;
                        }
                    }
                    const float ratio = ns > 0 ? __ldg(A.ratio + (size_t)q * M + s_em[j]) : 0.f;
                    for (int s = 0; s < ns; ++s) {
                        s_list[off + s] = make_int2(klo + TC_KV * s, j | (q << 9));
                        s_lw[off + s] = ratio;
                    }
                    off += ns;
                    atomicMax(&misc[MW_NLIST], (uint32_t)off);
                }
            }
            if (fold && tid < NB)
                tc_store_d(A, tmem + lane_d, accFull, n_commit & 1u, folded, true, s_abort, lane, b_first, 16 * G,
                           chunk, valid, nvox);
            if (fold) {
                ++n_commit;
                folded = true;
            }
            if (new_chain) chain0 = base;
            __syncthreads();  // the list is complete and D of an ended chain has been read
            if constexpr (CHAIN) tc_fence_after();
            const int n_list = (int)misc[MW_NLIST];
            const int p_next = (int)misc[MW_NEXT];

            if (tid < NB) {
                // ---- builders: group `grp` writes the W rows of the bundles with index = grp mod G ----
                const uint32_t grp = (uint32_t)(tid >> 7);
                const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
                int last_j = -1;
                bool inside = false;
                float r = 0.f;
                int Rb = 0;
                bool pending = false;  // a stored bundle whose completion is not yet signalled
                uint32_t pend_ps = 0;
                const int nb = (n_list + (int)H - 1) / (int)H;  // bundles of this round
                for (int e2 = (int)((grp + (uint32_t)G - bbase % (uint32_t)G) % (uint32_t)G); e2 < nb && !stop;
                     e2 += G) {
                    const uint32_t ps = bps;  // W bundle stage of this bundle
                    const int e0 = e2 * (int)H, nh = min((int)H, n_list - e0);
                    for (int h = 0; h < nh; ++h) {
                        const int e = e0 + h;
                        const int2 ent = s_list[e];
                        const int j = ent.y & 511, q = (ent.y >> 9) & 127;
                        if (j != last_j) {
                            last_j = j;
                            const float4 G4 = s_eg[j];
                            const float4 Nn = s_en[j];
                            Rb = s_erb[j];
                            const float ex = G4.x + dx, ey = G4.y + dy, ez = G4.z + dz;
                            inside = valid;
                            if (A.thr >= 0.f) {
                                const float zax = fmaf(ex, Nn.x, fmaf(ey, Nn.y, ez * Nn.z));
                                const float cx = fmaf(ey, Nn.z, -ez * Nn.y), cy = fmaf(ez, Nn.x, -ex * Nn.z),
                                            cz = fmaf(ex, Nn.y, -ey * Nn.x);
                                const float rho2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
                                inside = inside && (zax > 0.f) && (rho2 <= A.thr * zax * zax);
                            }
                            const float d = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
                            const float num = fmaf(2.f, fmaf(G4.x, dx, fmaf(G4.y, dy, G4.z * dz)), dd);
                            r = Nn.w + A.a * __fdividef(num, d + G4.w);
                        }
                        const float f = r + s_t[q * TILE_N + vl];
                        const float fl = floorf(f);
                        const float al = f - fl;
                        const int k = s_tb[q] + Rb + (int)fl;
                        const bool act = inside && (unsigned)k <= (unsigned)(K - 2);
                        const int u = k - ent.x;
                        float w = has_w ? s_w[q * TILE_N + vl] : 1.f;
                        w *= s_lw[e];
                        // e^{i th a} directly (th a in [0, th]; the weights are rounded to
                        // 16 bits), and e^{-i th (1-a)} = e^{i th a} e^{-i th}
                        float sn, cs;
                        __sincosf(A.theta * al, &sn, &cs);
                        const float uhr = cs, uhi = sn;
                        const float ubr = cs * A.er - sn * A.ei, ubi = cs * A.ei + sn * A.er;
                        const float w0 = w * (1.f - al), w1 = w * al;
                        const uint32_t pr = pack2<BF16>(w0 * uhr, w1 * ubr);  // (Wr[u], Wr[u+1])
                        const uint32_t pi = pack2<BF16>(w0 * uhi, w1 * ubi);  // (Wi[u], Wi[u+1])
                        // the row: (value u, value u + 1) of each plane at 16-bit position u,
                        // zeros elsewhere, by byte permutes with the selectors of row u
                        const bool in = act && (unsigned)u < (unsigned)TC_KV;
                        const uint4 *sel = reinterpret_cast<const uint4 *>(s_sel + 8 * (in ? u : TC_KV));
                        const uint4 s0 = sel[0], s1 = sel[1];
                        const uint32_t sw[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
                        uint32_t v[16];
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            v[c] = __byte_perm(pr, 0u, sw[c]);
                            v[8 + c] = __byte_perm(pi, 0u, sw[c]);
                        }
                        if (h == 0) {
                            // the group's previous bundle has drained while v was built: signal it
                            tmem_st_wait();
                            tc_fence_before();
                            __syncwarp();
                            mbar_arrive_if(&fullA[pend_ps], pending && lane == 0);
                            pending = false;
                            // this bundle's W stages are free once the MMAs of their previous use completed
                            if (bpass > 0) {
                                const uint32_t par = (bpass - 1u) & 1u;
                                const bool ready = __all_sync(0xffffffffu, mbar_try_wait(&emptyA[ps], par));
                                if (!ready && !tc_wait_warp(&emptyA[ps], par, s_abort, A.err, tc_limit(A))) {
                                    stop = true;
                                    break;
                                }
                            }
                            tc_fence_after();
                        }
                        tmem_st16(tmem + lane_base + (uint32_t)n + TC_ACOLS * (ps * H + (uint32_t)h), v);
                    }
                    if (stop) break;
                    pending = true;
                    pend_ps = ps;
                    for (bps += G; bps >= pa_n; ++bpass) bps -= pa_n;
                }
                tmem_st_wait();
                tc_fence_before();
                __syncwarp();
                mbar_arrive_if(&fullA[pend_ps], pending && lane == 0);
            } else if (warp == NB / 32) {
                // ---- producer: window copies, nprod lanes; lane L takes the bundles
                // with global index = L mod nprod, whose ring slots are = L mod nprod
                // (the slot count is a multiple of it); one barrier per bundle ----
                if ((uint32_t)lane < nprod) {
                    const int nb = (n_list + (int)H - 1) / (int)H;
                    for (int e2 = (int)(((uint32_t)lane + nprod - bbase % nprod) % nprod); e2 < nb && !stop;
                         e2 += (int)nprod) {
                        const uint32_t gb = bbase + (uint32_t)e2;
                        if (b_pass > 0 && !tc_wait(&emptyB[b_slot], (b_pass - 1) & 1u, s_abort, A.err, tc_limit(A))) {
                            stop = true;
                            break;
                        }
                        const int e0 = e2 * (int)H, nh = min((int)H, n_list - e0);
                        mbar_arrive_expect_tx(&fullB[b_slot], stage_bytes * (uint32_t)nh);
                        for (int h = 0; h < nh; ++h) {
                            const int2 ent = s_list[e0 + h];
                            const int j = ent.y & 511, q = (ent.y >> 9) & 127;
                            tma_load_4d(sB + (size_t)(b_slot * H + (uint32_t)h) * stage_bytes, &zmap, 8 * ent.x, 0, 0,
                                        (int)(qm_base + (size_t)q * M + s_em[j]), &fullB[b_slot]);
                        }
                        tma_issued = gb + 1u;
                        b_slot += nprod;
                        if (b_slot >= pb_n) {
                            b_slot -= pb_n;
                            ++b_pass;
                        }
                    }
                }
            } else {
                // ---- MMA issuer ----
                if (lane == 0) {
                    const uint32_t idesc = tc_idesc(n, BF16);
                    const uint64_t bdesc0 = smem_desc(smem_addr(sB), 128, 512);
                    uint32_t done = 0;
                    // test hook (das_plan_set_wait_test): the first CTA's first
                    // wait is on a barrier nothing arrives on, so it runs out
                    if (A.probe && blockIdx.x == 0 && blockIdx.y == 0 && base == 0 && n_list > 0 &&
                        !tc_wait(probe, 0u, s_abort, A.err, tc_limit(A)))
                        stop = true;
                    const int nb = (n_list + (int)H - 1) / (int)H;
                    for (int e2 = 0; e2 < nb && !stop; ++e2) {
                        const uint32_t ps = mps, slot = b_slot;  // W bundle stage and window bundle slot
                        if (!tc_wait(&fullA[ps], mpass & 1u, s_abort, A.err, tc_limit(A)) ||
                            !tc_wait(&fullB[slot], b_pass & 1u, s_abort, A.err, tc_limit(A))) {
                            stop = true;
                            break;
                        }
                        if (++mps == pa_n) {
                            mps = 0;
                            ++mpass;
                        }
                        if (++b_slot == pb_n) {
                            b_slot = 0;
                            ++b_pass;
                        }
                        tc_fence_after();
                        const int e0 = e2 * (int)H, nh = min((int)H, n_list - e0);
                        for (int h = 0; h < nh; ++h) {
                            const uint32_t gi = base + (uint32_t)(e0 + h);  // global sub-item index
                            const uint32_t a_col = tmem + (uint32_t)n + TC_ACOLS * (ps * H + (uint32_t)h);
                            const uint64_t bdesc = bdesc0 + (uint64_t)(((slot * H + (uint32_t)h) * stage_bytes) >> 4);
                            // the first sub-item of a chain starts from zero
                            mma_ts(tmem, a_col, bdesc, idesc, (CHAIN ? gi != chain0 : gi > 0) ? 1u : 0u);
                            mma_ts(tmem, a_col + 8, bdesc + (256 >> 4), idesc, 1u);
                        }
                        // the bundle's W stages and window slots are free once these MMAs complete
                        mma_commit(&emptyA[ps]);
                        mma_commit(&emptyB[slot]);
                        done = base + (uint32_t)(e0 + nh);
                    }
                    if (done) misc[MW_ISSUED] = done;
                }
            }
            base += (uint32_t)n_list;
            bbase += (uint32_t)((n_list + (int)H - 1) / (int)H);
            p0 = p_next;
            __syncthreads();  // list and element records of this round no longer read
            stop = stop || *s_abort != 0u;
        }
    }

    const uint32_t issued = misc[MW_ISSUED];  // written by the MMA thread before the last barrier
    if (warp == NB / 32 + 1 && lane == 0) {
        if (issued > chain0) mma_commit(accFull);
        if (issued > 0) atomicAdd(A.items, (unsigned long long)issued);
    }

    if (tid < NB) {
        // ---- epilogue: the last chain's D (TMEM) -> image ----
        if constexpr (CHAIN) {
            if (issued > chain0 || !folded)
                tc_store_d(A, tmem + lane_d, accFull, n_commit & 1u, folded, issued > chain0, s_abort, lane, b_first,
                           16 * G, chunk, valid, nvox);
        } else {
            // one chain: x = D smax; the groups take alternate 16-frame blocks.
            // MMAs still in flight must land before the tensor memory is read
            // or released, so this wait ignores aborts and is bounded by time only.
            bool ok = true;
            if (issued > 0 && lane == 0) {
                const uint64_t t0 = global_ns();
                while (!(ok = tc_try(accFull, 0u)))
                    if (global_ns() - t0 > TC_WAIT_NS) break;
                if (!ok) atomicOr(A.err, 4);
            }
            ok = __shfl_sync(0xffffffffu, ok, 0) != 0 && *s_abort == 0u;
            __syncwarp();
            tc_fence_after();
            const float sm = *A.smax;
            for (int b0 = b_first; b0 < A.bc; b0 += 16 * G) {
                uint32_t re[16], im[16];
                if (issued > 0) {
                    tmem_ld16(tmem + lane_d + (uint32_t)b0, re);
                    tmem_ld16(tmem + lane_d + (uint32_t)(A.bc + b0), im);
                    tmem_ld_wait();
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) re[i] = im[i] = 0u;
                }
                if (ok && valid) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int b = b0 + i;
                        const long long frame = (long long)chunk * A.bc + b;
                        if (b < A.bc && frame < A.B)
                            A.x[frame * g.n_voxels + nvox] =
                                make_float2(__uint_as_float(re[i]) * sm, __uint_as_float(im[i]) * sm);
                    }
                }
            }
            tc_fence_before();
        }
    } else if (warp == NB / 32 && (uint32_t)lane < nprod && *s_abort != 0u && tma_issued > 0) {
        // copies this lane still has in flight land before the CTA leaves:
        // wait for its last bundles of the ring (bounded by time)
        const uint64_t t0 = global_ns();
        uint32_t i = tma_issued - 1u;
        for (uint32_t c = 0; c < pb_n / nprod; ++c) {
            while (!tc_try(&fullB[i % pb_n], (i / pb_n) & 1u))
                if (global_ns() - t0 > TC_WAIT_NS) break;
            if (i < nprod) break;
            i -= nprod;
        }
    }
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, (uint32_t)A.ncols);
    }
}

// ---------------------------------------------------------------------------
// staging: scale ratios and the operand layout of the channel data
// ---------------------------------------------------------------------------

// Splits each (q, m) scale s between the two 16-bit operands: the samples are
// stored times zinv = 1 / sqrt(s smax) (at most sqrt(s / smax) <= 1 in
// magnitude) and the weights carry ratio = sqrt(s / smax), so neither operand
// falls into the f16 subnormal range for quiet channels; ratio * zinv =
// 1 / smax, and *smax = max(s) rescales the accumulator.  One block.
__global__ void __launch_bounds__(1024) tc_ratio_kernel(const float *__restrict__ scale, float *__restrict__ ratio,
                                                        float *__restrict__ zinv, float *__restrict__ smax, int QM) {
    __shared__ float red[32];
    float mx = 0.f;
    for (int i = threadIdx.x; i < QM; i += blockDim.x) mx = fmaxf(mx, scale[i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
    for (int i = threadIdx.x; i < QM; i += blockDim.x) {
        ratio[i] = sqrtf(scale[i] / mx);
        zinv[i] = 1.f / sqrtf(scale[i] * mx);
    }
    if (threadIdx.x == 0) *smax = mx;
}

// One thread per sample row k of one (chunk, q m): builds the n values of both
// planes, eight at a time, each written as one 16-byte vector.
template <bool BF16>
__global__ void __launch_bounds__(128) tc_relayout_kernel(const float2 *__restrict__ y, uint4 *__restrict__ z,
                                                          const float2 *__restrict__ rot,
                                                          const float *__restrict__ zinv, int B, int bc, int n,
                                                          int QM, int K) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.z;
    if (k >= K) return;
    const float2 r = rot ? rot[k] : make_float2(1.f, 0.f);
    const int nh = n >> 3;
    for (int qm = blockIdx.y; qm < QM; qm += gridDim.y) {
        const float s = zinv[qm];
        for (int h = 0; h < nh; ++h) {
            uint32_t p[4], q[4];
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
                float pv[2], qv[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int col = 8 * h + i + e;
                    const int f = col < bc ? col : col - bc;
                    const long long b = (long long)c * bc + f;
                    float2 v = make_float2(0.f, 0.f);
                    if (col < 2 * bc && f < bc && b < B) {
                        const float2 yv = y[((size_t)b * QM + qm) * (size_t)K + k];
                        v = make_float2((yv.x * r.x - yv.y * r.y) * s, (yv.x * r.y + yv.y * r.x) * s);
                    }
                    // plane 0: [Zr | Zi], plane 1: [-Zi | Zr]
                    pv[e] = col < bc ? v.x : v.y;
                    qv[e] = col < bc ? -v.y : v.x;
                }
                p[i >> 1] = pack2<BF16>(pv[0], pv[1]);
                q[i >> 1] = pack2<BF16>(qv[0], qv[1]);
            }
            const size_t row = (((size_t)c * QM + qm) * nh + h) * 2;
            z[row * K + k] = make_uint4(p[0], p[1], p[2], p[3]);
            z[(row + 1) * K + k] = make_uint4(q[0], q[1], q[2], q[3]);
        }
    }
}

void tc_shape(int B, int max_bc, int &bc, int &nch, int &n) {
    nch = (B + max_bc - 1) / max_bc;
    bc = (B + nch - 1) / nch;
    n = ((2 * bc + 15) / 16) * 16;
}

cudaError_t launch_tc_stage(const void *y, void *z, const float2 *rot, const float *scale, float *zinv,
                            float *ratio, float *smax, int bf16, int B, int bc, int nch, int n, int QM, int K,
                            cudaStream_t s) {
    tc_ratio_kernel<<<1, 1024, 0, s>>>(scale, ratio, zinv, smax, QM);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid((K + 127) / 128, QM < 65535 ? QM : 65535, nch);
    if (bf16)
        tc_relayout_kernel<true><<<grid, 128, 0, s>>>((const float2 *)y, (uint4 *)z, rot, zinv, B, bc, n, QM, K);
    else
        tc_relayout_kernel<false><<<grid, 128, 0, s>>>((const float2 *)y, (uint4 *)z, rot, zinv, B, bc, n, QM, K);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launch
// ---------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

template <bool BF16, int G, int MINB>
static cudaError_t launch_tc_t(const CUtensorMap &map, const TcArgs &A, size_t smem, int nch, cudaStream_t s) {
    auto kern = A.chain > 0 ? (A.hand == 2 ? tc_kernel<BF16, G, MINB, true, 2> : tc_kernel<BF16, G, MINB, true, 1>)
                            : (A.hand == 2 ? tc_kernel<BF16, G, MINB, false, 2> : tc_kernel<BF16, G, MINB, false, 1>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)n_tiles(A.g), (unsigned)nch);
    kern<<<grid, tc_threads(G), smem, s>>>(map, A);
    return cudaGetLastError();
}

cudaError_t launch_tc(const TcArgs &args, int bf16, const void *z, int nch, int ctas_per_sm, cudaStream_t s) {
    TcArgs A = args;
    if (A.n < 16 || A.n > 256 || A.n % 16 != 0 || A.bc < 1 || 2 * A.bc > A.n) return cudaErrorInvalidValue;
    if (((uintptr_t)z & 15u) != 0) return cudaErrorInvalidValue;
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return cudaErrorNotSupported;
    // CTAs per SM: automatically four CTAs of one builder group each while the
    // accumulator and two W stages fit 128 tensor-memory columns (N <= 96, up
    // to 48 frames) and the CTA's tables and window stages fit a quarter of the
    // shared memory, so that four MMA-issuing threads per SM overlap their
    // per-sub-item hand-offs (paper workload, 20 frames: 112.5 ms against
    // 137.3 ms with two CTAs); else two while they fit half of the tensor
    // memory and of the shared memory, else one.  Three, or the others, on
    // request (refused when they do not fit).
    const bool has_w = A.w_tx != nullptr;
    int G = 0, eb = 0, sbv = 0;
    // Fills the launch shape for `ps` CTAs per SM; false when it does not fit.
    auto configure = [&](int ps) -> bool {
        if (ps >= 3 && A.n + 2 * TC_ACOLS > 128) return false;
        if (ps == 2 && A.n + 2 * TC_ACOLS > 256) return false;
        A.ncols = ps >= 3 ? 128 : 512 / ps;
        // W stages: as many as the columns left beside the accumulator hold
        int sa = (A.ncols - A.n) / TC_ACOLS;
        if (sa > TC_MAX_SA) sa = TC_MAX_SA;
        if (sa < 2) return false;
        A.sa = sa;
        G = ps >= 3 ? 1 : ps == 2 ? 2 : 4;
        eb = G * TILE_N;
        // a list holds every sub-item of a block when no item needs two windows
        long long cap = (long long)eb * A.Q;
        if (cap < 256) cap = 256;
        if (cap > TC_LIST_MAX) cap = TC_LIST_MAX;
        // a chain ends at a list end: lists no longer than a chain keep chains short
        if (A.chain > 0 && cap > A.chain) cap = A.chain < 256 ? 256 : A.chain;
        A.list_cap = (int)cap;
        const size_t budget = (size_t)(227 * 1024) / ps - 1024;  // per-CTA share incl. the runtime's reserve
        const size_t fixed = tc_smem_layout(0, A.n, A.Q, has_w, eb, A.list_cap).total;
        const size_t stage = (size_t)64 * A.n;
        sbv = fixed < budget ? (int)((budget - fixed) / stage) : 0;
        if (sbv > TC_MAX_SB) sbv = TC_MAX_SB;
        sbv -= sbv % TC_PRODUCERS;
        if (sbv < TC_PRODUCERS) return false;
        // sub-items per hand-off: two while the W ring holds two bundles and at
        // least G (a group's wait on a stage is then at most one phase ahead of
        // it); paper workload, 20 frames, four CTAs per SM: 112.5 ms against
        // 118.1 ms with single sub-items
        int H = sa / 2 >= 2 && sa / 2 >= G ? 2 : 1;
        if (sa / H < G) return false;
        A.hand = H;
        A.sa = (sa / H) * H;
        return true;
    };
    int per_sm = 0;
    if (ctas_per_sm > 0) {
        per_sm = ctas_per_sm > 4 ? 4 : ctas_per_sm;
        if (!configure(per_sm)) {  // keep the former fallback of an explicit request to fewer CTAs
            if (per_sm >= 3 && configure(2)) per_sm = 2;
            else if (per_sm >= 2 && configure(1)) per_sm = 1;
            else return cudaErrorInvalidConfiguration;
        }
    } else {
        const int tries[3] = {4, 2, 1};
        for (int ps : tries)
            if (configure(ps)) { per_sm = ps; break; }
        if (per_sm == 0) return cudaErrorInvalidConfiguration;
    }
    A.sb = sbv;
    const size_t smem = tc_smem_layout(sbv, A.n, A.Q, has_w, eb, A.list_cap).total;

    // The window of one item is, for every (column group, plane), 16 rows x
    // 8 values contiguous in memory: the map merges (row, 8 values) into one
    // 4-D dimension, so a box moves 256-byte runs; its x coordinate 8 k0 is
    // always 16-byte aligned and rows outside 0 .. K-1 arrive as zeros.
    CUtensorMap map;
    const int QM = A.Q * A.M;
    const cuuint64_t dims[4] = {(cuuint64_t)A.K * 8, 2, (cuuint64_t)(A.n / 8), (cuuint64_t)nch * QM};
    const cuuint64_t strides[3] = {(cuuint64_t)A.K * 16, (cuuint64_t)A.K * 32, (cuuint64_t)(A.n / 8) * A.K * 32};
    const cuuint32_t box[4] = {(cuuint32_t)TC_U * 8, 2, (cuuint32_t)(A.n / 8), 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(&map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4,
                              const_cast<void *>(z), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    if (per_sm == 4) {
        return bf16 ? launch_tc_t<true, 1, 4>(map, A, smem, nch, s) : launch_tc_t<false, 1, 4>(map, A, smem, nch, s);
    }
    if (per_sm == 3) {
        return bf16 ? launch_tc_t<true, 1, 3>(map, A, smem, nch, s) : launch_tc_t<false, 1, 3>(map, A, smem, nch, s);
    }
    if (per_sm == 2) {
        return bf16 ? launch_tc_t<true, 2, 2>(map, A, smem, nch, s) : launch_tc_t<false, 2, 2>(map, A, smem, nch, s);
    }
    return bf16 ? launch_tc_t<true, 4, 1>(map, A, smem, nch, s) : launch_tc_t<false, 4, 1>(map, A, smem, nch, s);
}

}  // namespace das
