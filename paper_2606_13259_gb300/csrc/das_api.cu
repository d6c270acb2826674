// das_api.cu -- the C-ABI of include/das.h: plan construction (geometry to the
// device, per-tile transmit tables), argument checking, scratch management and
// kernel dispatch.  See das.h for the contract of every entry point.
#include "das.h"
#include "das_internal.cuh"
#include "das_tc.cuh"

#include <sys/mman.h>
#include <unistd.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

using namespace das;

static thread_local char g_err[1024];

constexpr int HOST_COPY_STREAMS = 16;

// mappings behind the pointers das_host_alloc returned
struct HostMap {
    void *base;
    size_t len;
};
static std::mutex g_host_mutex;
static std::map<void *, HostMap> g_host_maps;

static int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

static int cuda_fail(cudaError_t e, const char *what) {
    const int code = (e == cudaErrorMemoryAllocation) ? DAS_ERR_OOM : DAS_ERR_CUDA;
    return fail(code, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define DAS_CU(call)                                                 \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);          \
    } while (0)

struct das_plan {
    int device = 0;
    GridDesc g{};
    int M = 0, Q = 0, K = 0;
    int sample_type = 0, storage = 0, max_batch = 1, t0_offset = 1;
    double c = 0, fs = 0, f_demod = 0, f_number = 0;
    double t0[3] = {0, 0, 0};
    bool has_w = false;
    double *elem_pos = nullptr;
    float4 *elem_nrm = nullptr;
    int *tx_kind = nullptr;
    double *tx_vec = nullptr;
    double *tx_off = nullptr;
    int *tx_tb = nullptr;
    float *tx_t = nullptr;
    float *tx_tmin = nullptr;
    float *tx_tmax = nullptr;
    int2 *tx_span = nullptr;
    int *err = nullptr;
    float *w_tx = nullptr;
    float2 *rot = nullptr;
    float *scale = nullptr;
    float *inv_scale = nullptr;
    void *z = nullptr;
    size_t z_bytes = 0;
    double *partial = nullptr;
    size_t partial_n = 0;
    double *scalar = nullptr;
    void *stage_y[2] = {nullptr, nullptr};  // host calls: device staging of inputs / images
    void *stage_x[2] = {nullptr, nullptr};  //   (slot 1 only for the overlapped sequence call)
    std::vector<cudaStream_t> copy_streams;  // host calls: copies split across these
    std::vector<cudaEvent_t> copy_events;    // [0] start, [1 + i] end of stream i
    // overlapped sequence call, per staging slot: ends of the input pieces,
    // ends of the image pieces, end of the forward pass
    std::vector<cudaEvent_t> in_done[2], out_done[2];
    cudaEvent_t fwd_done[2] = {nullptr, nullptr};
    void *z_tc = nullptr;      // tensor-core operand layout of the channel data
    size_t z_tc_bytes = 0;
    float *ratio = nullptr;    // [Q][M] scale / largest scale (tensor-core path)
    float *smax = nullptr;     // largest scale (tensor-core path)
    unsigned long long *tc_items = nullptr;  // MMA sub-items issued (tensor-core path)
    int tc_n = 0;              // MMA N of the last tensor-core call
    bool dirty = true;
    unsigned long long wait_ns = 0;  // test hook: limit of the kernels' pipeline waits (0: 1 s)
    int wait_probe = 0;              // test hook: one CTA waits on a barrier nothing arrives on
    das_tuning_t tuning{};
    size_t bytes = 0;
    long long launches = 0;
    std::vector<cudaEvent_t> ev_start, ev_stop;
    int ev_used = 0;
    std::vector<void *> allocs;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int dalloc(das_plan *p, void **ptr, size_t bytes, const char *what) {
    *ptr = nullptr;
    if (bytes == 0) return DAS_OK;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? DAS_ERR_OOM : DAS_ERR_CUDA, "cudaMalloc(%zu bytes) for %s: %s",
                    bytes, what, cudaGetErrorString(e));
    }
    p->allocs.push_back(*ptr);
    p->bytes += bytes;
    return DAS_OK;
}

// Frees one of the plan's buffers after the device has finished all work that
// may still read it.
void dfree(das_plan *p, void *ptr) {
    if (!ptr) return;
    cudaDeviceSynchronize();
    for (size_t i = 0; i < p->allocs.size(); ++i)
        if (p->allocs[i] == ptr) { p->allocs.erase(p->allocs.begin() + i); break; }
    cudaFree(ptr);
}

bool is_iq(const das_plan *p) { return p->sample_type == DAS_SAMPLE_C64; }

int sample_bytes_public(const das_plan *p) { return is_iq(p) ? 8 : 4; }

int sample_bytes_store(const das_plan *p) {
    const int comp = is_iq(p) ? 2 : 1;
    return comp * (p->storage == DAS_STORE_F32 ? 4 : (p->storage == DAS_STORE_E4M3 || p->storage == DAS_STORE_E5M2) ? 1 : 2);
}

const int FB_F32[] = {20, 16, 12, 8, 4, 2, 1};
constexpr int ADJ_ROWS = 256;  // sample rows per adjoint CTA (das_adjoint.cu); measured best of 32..K
const int FB_16[] = {24, 20, 16, 12, 8, 4, 2, 1};

// Frames per thread for a call with B frames: the supported value minimising
// chunks * (geometry overhead + frames per chunk), ties to the larger.
int choose_fb(const das_plan *p, int B, int mode) {
    const int store = p->storage;
    if (p->tuning.frames_per_thread > 0 && tile_fb_supported(mode, is_iq(p), store, p->tuning.frames_per_thread))
        return p->tuning.frames_per_thread;
    const int *list = (store == DAS_STORE_F32 || mode != MODE_FWD) ? FB_F32 : FB_16;
    const int nl = (store == DAS_STORE_F32 || mode != MODE_FWD) ? 7 : 8;
    const int overhead = 6;
    int best = 1;
    long best_cost = -1;
    for (int i = 0; i < nl; ++i) {
        const int fb = list[i];
        if (!tile_fb_supported(mode, is_iq(p), store, fb)) continue;
        const long chunks = (B + fb - 1) / fb;
        const long cost = chunks * (overhead + fb);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = fb; }
    }
    return best;
}

int padded_batch(const das_plan *p, int B, int mode) {
    const int fb = choose_fb(p, B, mode);
    return ((B + fb - 1) / fb) * fb;
}

size_t scratch_bytes_for(const das_plan *p) {
    int bs = 1;
    for (int B = 1; B <= p->max_batch; ++B) {
        const int a = padded_batch(p, B, MODE_FWD);
        const int b = p->storage == DAS_STORE_F32 ? padded_batch(p, B, MODE_DC) : 1;
        bs = a > bs ? a : bs;
        bs = b > bs ? b : bs;
    }
    return (size_t)p->Q * p->M * p->K * (size_t)bs * sample_bytes_store(p);
}

int ensure_scratch(das_plan *p) {
    const size_t need = scratch_bytes_for(p);
    if (need <= p->z_bytes) return DAS_OK;
    dfree(p, p->z);
    p->bytes -= p->z_bytes;
    p->z = nullptr;
    p->z_bytes = 0;
    int rc = dalloc(p, &p->z, need, "channel-data scratch");
    if (rc != DAS_OK) return rc;
    p->z_bytes = need;
    return DAS_OK;
}

int prepare_if_dirty(das_plan *p, cudaStream_t s) {
    if (!p->dirty) return DAS_OK;
    DAS_CU(launch_prepare(p->g, p->Q, p->tx_kind, p->tx_vec, p->tx_off, p->t0, p->fs / p->c, p->tx_tb, p->tx_t,
                          p->tx_tmin, p->tx_tmax, p->tx_span, s));
    p->launches += 1;
    p->dirty = false;
    return DAS_OK;
}

void destroy_events(das_plan *p) {
    for (cudaEvent_t e : p->ev_start) cudaEventDestroy(e);
    for (cudaEvent_t e : p->ev_stop) cudaEventDestroy(e);
    p->ev_start.clear();
    p->ev_stop.clear();
    p->ev_used = 0;
}

void fill_common(const das_plan *p, float &a, double &ad, float &theta, float &hr, float &hi, float &thr, float &rad) {
    ad = p->fs / p->c;
    a = (float)ad;
    const double th = 2.0 * M_PI * p->f_demod / p->fs;
    theta = (float)th;
    hr = (float)cos(0.5 * th);
    hi = (float)sin(0.5 * th);
    thr = p->f_number > 0 ? (float)((1.0 + 1e-6) / (4.0 * p->f_number * p->f_number)) : -1.f;
    const double rx = 0.5 * (TILE_X - 1) * p->g.sx, ry = 0.5 * (TILE_Y - 1) * p->g.sy,
                 rz = 0.5 * (TILE_Z - 1) * p->g.sz;
    rad = (float)(sqrt(rx * rx + ry * ry + rz * rz) * (1.0 + 1e-4) + 1e-9);
}

TileArgs tile_args(const das_plan *p, int B, int fb, const void *z) {
    TileArgs A{};
    A.g = p->g;
    A.M = p->M;
    A.Q = p->Q;
    A.K = p->K;
    A.B = B;
    A.fb = fb;
    fill_common(p, A.a, A.ad, A.theta, A.hr, A.hi, A.thr, A.tile_radius);
    const double aR = (p->fs / p->c) * (double)A.tile_radius;
    A.umax = p->tuning.staging ? window_rows(aR) : 0;
    A.w256 = p->tuning.load_width == 256 ? 1 : 0;
    A.win_lo = (float)(aR + 1e-3);
    A.tx_tmin = p->tx_tmin;
    A.err = p->err;
    A.wait_ns = p->wait_ns;
    A.probe = p->wait_probe;
    A.inv_c = 1.0 / p->c;
    A.elem_pos = p->elem_pos;
    A.elem_nrm = p->elem_nrm;
    A.tx_tb = p->tx_tb;
    A.tx_t = p->tx_t;
    A.w_tx = p->w_tx;
    A.scale = p->storage == DAS_STORE_F32 ? nullptr : p->scale;
    A.z = z;
    return A;
}

bool aligned(const void *ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

// Whether the tile kernels of a call with `fb` frames per thread read the
// relayouted rows in column order (LD_COL in das_tile.cuh): the default load
// path, unless a tuning asks for staged windows or a fixed row load width.
int col_layout(const das_plan *p, int fb) {
    return (!p->tuning.staging && p->tuning.load_width == 0 && tile_col_supported(is_iq(p), p->storage, fb)) ? 1 : 0;
}

// Relayout of the public channel data into the plan scratch (or the data
// itself when the layouts coincide), in column order when `col`.  Returns the
// pointer the kernels read.
int stage_channels(das_plan *p, const void *y, int B, int fb, int nch, int col, cudaStream_t s, const void **z_out) {
    const int Bs = fb * nch;
    const bool iq = is_iq(p);
    const int QM = p->Q * p->M;
    if (p->storage != DAS_STORE_F32) {
        DAS_CU(launch_scale(y, p->scale, p->inv_scale, iq, p->storage, B, QM, p->K, s));
        p->launches += 1;
    }
    if (!iq && p->storage == DAS_STORE_F32 && Bs == 1 && !col) {
        *z_out = y;
        return DAS_OK;
    }
    const size_t need = (size_t)QM * p->K * (size_t)Bs * sample_bytes_store(p);
    if (need > p->z_bytes) return fail(DAS_ERR_INVALID_ARG, "batch needs %zu bytes of scratch, plan holds %zu", need, p->z_bytes);
    DAS_CU(launch_relayout(y, p->z, iq ? p->rot : nullptr, p->storage == DAS_STORE_F32 ? nullptr : p->inv_scale, iq,
                           p->storage, B, fb, nch, QM, p->K, col, s));
    p->launches += 1;
    *z_out = p->z;
    return DAS_OK;
}

bool tc_capable(const das_plan *p) {
    return is_iq(p) && (p->storage == DAS_STORE_F16 || p->storage == DAS_STORE_BF16);
}

// Operand scratch of the tensor-core path: chunks x (q, m) x n columns x K
// rows x 2 planes x 2 bytes, the largest over the batch sizes the plan takes.
size_t tc_scratch_bytes(const das_plan *p) {
    size_t best = 0;
    for (int B = 1; B <= p->max_batch; ++B) {
        int bc, nch, n;
        tc_shape(B, tc_max_frames(p->tuning.ctas_per_sm), bc, nch, n);
        const size_t b = (size_t)nch * p->Q * p->M * (size_t)n * p->K * 4;
        best = b > best ? b : best;
    }
    return best;
}

int ensure_tc_scratch(das_plan *p) {
    int rc;
    if (!p->ratio && (rc = dalloc(p, (void **)&p->ratio, sizeof(float) * (size_t)p->Q * p->M, "scale ratios")) != DAS_OK)
        return rc;
    if (!p->smax && (rc = dalloc(p, (void **)&p->smax, sizeof(float), "largest scale")) != DAS_OK) return rc;
    if (!p->tc_items) {
        if ((rc = dalloc(p, (void **)&p->tc_items, sizeof(unsigned long long), "MMA item counter")) != DAS_OK) return rc;
        DAS_CU(cudaMemset(p->tc_items, 0, sizeof(unsigned long long)));
    }
    const size_t need = tc_scratch_bytes(p);
    if (need <= p->z_tc_bytes) return DAS_OK;
    dfree(p, p->z_tc);
    p->bytes -= p->z_tc_bytes;
    p->z_tc = nullptr;
    p->z_tc_bytes = 0;
    if ((rc = dalloc(p, &p->z_tc, need, "tensor-core operand scratch")) != DAS_OK) return rc;
    p->z_tc_bytes = need;
    return DAS_OK;
}

// Forward pass on the tensor cores: per-(q, m) scales, the operand relayout,
// then the tcgen05 kernel (das_tc.cu).  `timing`: record the plan's kernel
// events when they are enabled (not inside a batch's graph capture).
int forward_tc(das_plan *p, const void *y, void *x, int B, cudaStream_t s, bool timing = true) {
    int bc, nch, n;
    tc_shape(B, tc_max_frames(p->tuning.ctas_per_sm), bc, nch, n);
    const int QM = p->Q * p->M;
    const size_t need = (size_t)nch * QM * (size_t)n * p->K * 4;
    if (need > p->z_tc_bytes || !p->ratio || !p->smax)
        return fail(DAS_ERR_INVALID_ARG, "tensor-core scratch holds %zu bytes, batch needs %zu", p->z_tc_bytes, need);
    const bool bf16 = p->storage == DAS_STORE_BF16;
    DAS_CU(launch_scale(y, p->scale, p->inv_scale, 1, p->storage, B, QM, p->K, s));
    // the samples' factors go to inv_scale (scratch of the CUDA-core path, refilled there on every call)
    DAS_CU(launch_tc_stage(y, p->z_tc, p->rot, p->scale, p->inv_scale, p->ratio, p->smax, bf16 ? 1 : 0, B, bc, nch, n,
                           QM, p->K, s));
    p->launches += 3;
    TcArgs A{};
    A.g = p->g;
    A.M = p->M;
    A.Q = p->Q;
    A.K = p->K;
    A.B = B;
    A.bc = bc;
    A.n = n;
    fill_common(p, A.a, A.ad, A.theta, A.hr, A.hi, A.thr, A.tile_radius);
    A.er = (float)cos(2.0 * M_PI * p->f_demod / p->fs);
    A.ei = (float)-sin(2.0 * M_PI * p->f_demod / p->fs);
    A.ahx = (float)(A.ad * 0.5 * (TILE_X - 1) * p->g.sx);
    A.ahy = (float)(A.ad * 0.5 * (TILE_Y - 1) * p->g.sy);
    A.ahz = (float)(A.ad * 0.5 * (TILE_Z - 1) * p->g.sz);
    A.aR = (float)(A.ad * A.tile_radius);
    A.aR2h = (float)(A.ad * (double)A.tile_radius * A.tile_radius * 0.5);
    A.elem_pos = p->elem_pos;
    A.elem_nrm = p->elem_nrm;
    A.tx_tb = p->tx_tb;
    A.tx_t = p->tx_t;
    A.tx_tmin = p->tx_tmin;
    A.tx_tmax = p->tx_tmax;
    A.w_tx = p->w_tx;
    A.ratio = p->ratio;
    A.smax = p->smax;
    A.err = p->err;
    A.wait_ns = p->wait_ns;
    A.probe = p->wait_probe;
    A.items = p->tc_items;
    A.x = reinterpret_cast<float2 *>(x);
    A.chain = p->tuning.tc_chain > 0 ? p->tuning.tc_chain
              : (p->tuning.tc_chain == 0 && p->Q >= TC_CHAIN_MIN_TX ? TC_CHAIN_DEFAULT : 0);
    p->tc_n = n;
    const bool timed = timing && p->ev_used < (int)p->ev_start.size();
    if (timed) DAS_CU(cudaEventRecord(p->ev_start[p->ev_used], s));
    DAS_CU(launch_tc(A, bf16 ? 1 : 0, p->z_tc, nch, p->tuning.ctas_per_sm, s));
    p->launches += 1;
    if (timed) {
        DAS_CU(cudaEventRecord(p->ev_stop[p->ev_used], s));
        p->ev_used += 1;
    }
    return DAS_OK;
}

// Copies `bytes` between host and device as HOST_COPY_STREAMS pieces on the
// plan's copy streams, ordered after the work already queued on `s` and
// before what follows on it.  Host pages that the GPU's address translation
// lost during long kernels are fetched by many copy engines at once instead
// of one.
int copy_split(das_plan *p, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s) {
    const size_t min_piece = (size_t)16 << 20;
    int pieces = (int)((bytes + min_piece - 1) / min_piece);
    if (pieces > HOST_COPY_STREAMS) pieces = HOST_COPY_STREAMS;
    if (pieces <= 1) {
        DAS_CU(cudaMemcpyAsync(dst, src, bytes, kind, s));
        return DAS_OK;
    }
    const size_t piece = ((bytes + pieces - 1) / pieces + 255) / 256 * 256;
    DAS_CU(cudaEventRecord(p->copy_events[0], s));
    for (int i = 0; i < pieces; ++i) {
        const size_t off = (size_t)i * piece;
        if (off >= bytes) break;
        const size_t len = off + piece <= bytes ? piece : bytes - off;
        cudaStream_t cs = p->copy_streams[i];
        DAS_CU(cudaStreamWaitEvent(cs, p->copy_events[0], 0));
        DAS_CU(cudaMemcpyAsync((char *)dst + off, (const char *)src + off, len, kind, cs));
        DAS_CU(cudaEventRecord(p->copy_events[1 + i], cs));
        DAS_CU(cudaStreamWaitEvent(s, p->copy_events[1 + i], 0));
    }
    return DAS_OK;
}

}  // namespace

extern "C" {

const char *das_last_error(void) { return g_err; }

const char *das_version(void) { return "das-gb300 0.1.0 (sm_103a)"; }

int das_plan_create(das_plan_t **out, const das_geometry_t *geometry, const das_grid_t *grid,
                    const das_tx_t *tx_list, int n_tx, double c, double fs, double f_demod, double f_number,
                    const das_options_t *options) {
    g_err[0] = 0;
    if (!out) return fail(DAS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!geometry || !grid || !tx_list || !options) return fail(DAS_ERR_INVALID_ARG, "NULL argument");
    if (geometry->n_elements < 1 || !geometry->positions) return fail(DAS_ERR_INVALID_ARG, "need >= 1 element with positions");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return fail(DAS_ERR_INVALID_ARG, "grid dimensions must be >= 1");
    for (int i = 0; i < 3; ++i)
        if (!(grid->spacing[i] > 0) || !std::isfinite(grid->spacing[i]) || !std::isfinite(grid->origin[i]))
            return fail(DAS_ERR_INVALID_ARG, "grid spacing must be positive and finite");
    if (n_tx < 1) return fail(DAS_ERR_INVALID_ARG, "need >= 1 transmit");
    if (n_tx > 128) return fail(DAS_ERR_UNSUPPORTED, "at most 128 transmits per plan (got %d)", n_tx);
    if (!(c > 0) || !std::isfinite(c)) return fail(DAS_ERR_INVALID_ARG, "c must be positive");
    if (!(fs > 0) || !std::isfinite(fs)) return fail(DAS_ERR_INVALID_ARG, "fs must be positive");
    if (!(f_demod >= 0) || !std::isfinite(f_demod)) return fail(DAS_ERR_INVALID_ARG, "f_demod must be >= 0");
    if (!std::isfinite(f_number)) return fail(DAS_ERR_INVALID_ARG, "f_number must be finite");
    if (options->n_samples < 2) return fail(DAS_ERR_INVALID_ARG, "n_samples must be >= 2");
    if (options->sample_type != DAS_SAMPLE_F32 && options->sample_type != DAS_SAMPLE_C64)
        return fail(DAS_ERR_INVALID_ARG, "unknown sample_type %d", options->sample_type);
    if (options->storage < DAS_STORE_F32 || options->storage > DAS_STORE_E5M2)
        return fail(DAS_ERR_INVALID_ARG, "unknown storage %d", options->storage);
    if ((options->storage == DAS_STORE_E4M3 || options->storage == DAS_STORE_E5M2) &&
        options->sample_type != DAS_SAMPLE_C64)
        return fail(DAS_ERR_UNSUPPORTED, "8-bit storage is provided for IQ data only");
    if (options->max_batch < 1) return fail(DAS_ERR_INVALID_ARG, "max_batch must be >= 1");
    if (options->sample_type == DAS_SAMPLE_F32 && f_demod != 0.0)
        return fail(DAS_ERR_INVALID_ARG, "real RF data (DAS_SAMPLE_F32) need f_demod = 0");
    const long long N = (long long)grid->nx * grid->ny * grid->nz;
    if (N > (1LL << 40)) return fail(DAS_ERR_UNSUPPORTED, "grid too large");

    for (int m = 0; m < geometry->n_elements; ++m) {
        double len2 = 0;
        for (int i = 0; i < 3; ++i) {
            if (!std::isfinite(geometry->positions[3 * m + i])) return fail(DAS_ERR_INVALID_ARG, "element %d position not finite", m);
            const double v = geometry->normals ? geometry->normals[3 * m + i] : (i == 2 ? 1.0 : 0.0);
            len2 += v * v;
        }
        if (!(fabs(sqrt(len2) - 1.0) <= 1e-6)) return fail(DAS_ERR_INVALID_ARG, "element %d normal is not a unit vector", m);
    }
    for (int q = 0; q < n_tx; ++q) {
        const int kd = tx_list[q].kind;
        if (kd < DAS_TX_DIVERGING || kd > DAS_TX_NONE) return fail(DAS_ERR_INVALID_ARG, "transmit %d: unknown kind %d", q, kd);
        double l2 = 0;
        for (int i = 0; i < 3; ++i) {
            if (!std::isfinite(tx_list[q].vec[i])) return fail(DAS_ERR_INVALID_ARG, "transmit %d: vector not finite", q);
            l2 += tx_list[q].vec[i] * tx_list[q].vec[i];
        }
        if (kd == DAS_TX_PLANE && !(fabs(sqrt(l2) - 1.0) <= 1e-6))
            return fail(DAS_ERR_INVALID_ARG, "transmit %d: plane direction is not a unit vector", q);
    }

    das_plan *p = new (std::nothrow) das_plan();
    if (!p) return fail(DAS_ERR_OOM, "host allocation failed");
    auto bail = [&](int rc) {
        for (void *a : p->allocs) cudaFree(a);
        delete p;
        return rc;
    };
    if (cudaGetDevice(&p->device) != cudaSuccess) { cudaGetLastError(); return bail(fail(DAS_ERR_CUDA, "no CUDA device")); }

    GridDesc &g = p->g;
    g.nx = grid->nx; g.ny = grid->ny; g.nz = grid->nz;
    g.tiles_x = (grid->nx + TILE_X - 1) / TILE_X;
    g.tiles_y = (grid->ny + TILE_Y - 1) / TILE_Y;
    g.tiles_z = (grid->nz + TILE_Z - 1) / TILE_Z;
    g.n_voxels = N;
    g.ox = grid->origin[0]; g.oy = grid->origin[1]; g.oz = grid->origin[2];
    g.sx = grid->spacing[0]; g.sy = grid->spacing[1]; g.sz = grid->spacing[2];
    if (n_tiles(g) > 0x7fffffffLL) return bail(fail(DAS_ERR_UNSUPPORTED, "too many voxel tiles"));
    p->M = geometry->n_elements;
    p->Q = n_tx;
    p->K = options->n_samples;
    p->sample_type = options->sample_type;
    p->storage = options->storage;
    p->max_batch = options->max_batch;
    p->t0_offset = options->t0_offset ? 1 : 0;
    p->c = c; p->fs = fs; p->f_demod = f_demod; p->f_number = f_number;
    for (int i = 0; i < 3; ++i) p->t0[i] = geometry->t0_ref[i];

    // host copies of the geometry
    const int M = p->M, Q = p->Q;
    std::vector<double> pos(3 * (size_t)M);
    std::vector<float4> nrm(M);
    for (int m = 0; m < M; ++m) {
        double n[3] = {0, 0, 1};
        for (int i = 0; i < 3; ++i) {
            pos[3 * m + i] = geometry->positions[3 * m + i];
            if (!std::isfinite(pos[3 * m + i])) return bail(fail(DAS_ERR_INVALID_ARG, "element %d position not finite", m));
            if (geometry->normals) n[i] = geometry->normals[3 * m + i];
        }
        const double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(len > 0) || fabs(len - 1.0) > 1e-6) return bail(fail(DAS_ERR_INVALID_ARG, "element %d normal is not a unit vector", m));
        nrm[m] = make_float4((float)n[0], (float)n[1], (float)n[2], 0.f);
    }
    std::vector<int> kind(Q);
    std::vector<double> vec(3 * (size_t)Q), off(Q, 0.0);
    for (int q = 0; q < Q; ++q) {
        kind[q] = tx_list[q].kind;
        if (kind[q] < DAS_TX_DIVERGING || kind[q] > DAS_TX_NONE) return bail(fail(DAS_ERR_INVALID_ARG, "transmit %d: unknown kind", q));
        for (int i = 0; i < 3; ++i) {
            vec[3 * q + i] = tx_list[q].vec[i];
            if (!std::isfinite(vec[3 * q + i])) return bail(fail(DAS_ERR_INVALID_ARG, "transmit %d: vector not finite", q));
        }
        if (kind[q] == DAS_TX_PLANE) {
            const double l = sqrt(vec[3 * q] * vec[3 * q] + vec[3 * q + 1] * vec[3 * q + 1] + vec[3 * q + 2] * vec[3 * q + 2]);
            if (fabs(l - 1.0) > 1e-6) return bail(fail(DAS_ERR_INVALID_ARG, "transmit %d: plane direction is not a unit vector", q));
        }
        if (kind[q] == DAS_TX_DIVERGING && p->t0_offset) {
            const double dx = vec[3 * q] - p->t0[0], dy = vec[3 * q + 1] - p->t0[1], dz = vec[3 * q + 2] - p->t0[2];
            off[q] = sqrt(dx * dx + dy * dy + dz * dz);
        }
        if (tx_list[q].w_tx) p->has_w = true;
    }

    const long long T = n_tiles(g);
    int rc;
    cudaError_t e0;
#define DAS_ALLOC(ptr, bytes, what) \
    if ((rc = dalloc(p, (void **)&(ptr), (bytes), (what))) != DAS_OK) return bail(rc)
    DAS_ALLOC(p->elem_pos, sizeof(double) * 3 * M, "element positions");
    DAS_ALLOC(p->elem_nrm, sizeof(float4) * M, "element normals");
    DAS_ALLOC(p->tx_kind, sizeof(int) * Q, "transmit kinds");
    DAS_ALLOC(p->tx_vec, sizeof(double) * 3 * Q, "transmit vectors");
    DAS_ALLOC(p->tx_off, sizeof(double) * Q, "transmit offsets");
    DAS_ALLOC(p->tx_tb, sizeof(int) * (size_t)T * Q, "transmit bases");
    DAS_ALLOC(p->tx_t, sizeof(float) * (size_t)T * Q * TILE_N, "transmit delays");
    DAS_ALLOC(p->tx_tmin, sizeof(float) * (size_t)T * Q, "transmit delay minima");
    DAS_ALLOC(p->tx_tmax, sizeof(float) * (size_t)T * Q, "transmit delay maxima");
    DAS_ALLOC(p->tx_span, sizeof(int2) * (size_t)T, "transmit row spans");
    DAS_ALLOC(p->err, sizeof(int), "device error word");
    if ((e0 = cudaMemset(p->err, 0, sizeof(int))) != cudaSuccess) return bail(cuda_fail(e0, "cudaMemset"));
    DAS_ALLOC(p->partial, sizeof(double) * (size_t)T * p->max_batch, "partials");
    DAS_ALLOC(p->scalar, sizeof(double), "scalar");
    p->partial_n = (size_t)T * p->max_batch;
    if (p->storage != DAS_STORE_F32) {
        DAS_ALLOC(p->scale, sizeof(float) * (size_t)Q * M, "storage scale");
        DAS_ALLOC(p->inv_scale, sizeof(float) * (size_t)Q * M, "storage inverse scale");
    }
    if (is_iq(p) && f_demod != 0.0) DAS_ALLOC(p->rot, sizeof(float2) * p->K, "rotation table");
    if ((rc = ensure_scratch(p)) != DAS_OK) return bail(rc);

    cudaError_t e;
#define DAS_UP(dst, src, bytes) \
    if ((e = cudaMemcpy((dst), (src), (bytes), cudaMemcpyHostToDevice)) != cudaSuccess) return bail(cuda_fail(e, "upload"))
    DAS_UP(p->elem_pos, pos.data(), sizeof(double) * 3 * M);
    DAS_UP(p->elem_nrm, nrm.data(), sizeof(float4) * M);
    DAS_UP(p->tx_kind, kind.data(), sizeof(int) * Q);
    DAS_UP(p->tx_vec, vec.data(), sizeof(double) * 3 * Q);
    DAS_UP(p->tx_off, off.data(), sizeof(double) * Q);
    if (p->rot) {
        // e^{i 2 pi (f_d / fs) k}, reduced to one turn in float64
        std::vector<float2> rot(p->K);
        const double ratio = f_demod / fs;
        for (int k = 0; k < p->K; ++k) {
            double turns = ratio * k;
            turns -= floor(turns);
            rot[k] = make_float2((float)cos(2.0 * M_PI * turns), (float)sin(2.0 * M_PI * turns));
        }
        DAS_UP(p->rot, rot.data(), sizeof(float2) * p->K);
    }
    if (p->has_w) {
        DAS_ALLOC(p->w_tx, sizeof(float) * (size_t)T * Q * TILE_N, "transmit weights");
        std::vector<float> w((size_t)T * Q * TILE_N, 0.f);
        for (long long t = 0; t < T; ++t) {
            const int tx = (int)(t % g.tiles_x), ty = (int)((t / g.tiles_x) % g.tiles_y),
                      tz = (int)(t / ((long long)g.tiles_x * g.tiles_y));
            for (int l = 0; l < TILE_N; ++l) {
                int lx, ly, lz;
                lane_offset(l, lx, ly, lz);
                const int ix = tx * TILE_X + lx, iy = ty * TILE_Y + ly, iz = tz * TILE_Z + lz;
                if (ix >= g.nx || iy >= g.ny || iz >= g.nz) continue;
                const long long n = ((long long)iz * g.ny + iy) * g.nx + ix;
                for (int q = 0; q < Q; ++q)
                    w[((size_t)t * Q + q) * TILE_N + l] = tx_list[q].w_tx ? tx_list[q].w_tx[n] : 1.f;
            }
        }
        DAS_UP(p->w_tx, w.data(), sizeof(float) * w.size());
    }
    rc = prepare_if_dirty(p, nullptr);
    if (rc != DAS_OK) return bail(rc);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(cuda_fail(e, "plan preparation"));
    *out = p;
    return DAS_OK;
#undef DAS_ALLOC
#undef DAS_UP
}

void das_plan_destroy(das_plan_t *plan) {
    if (!plan) return;
    DeviceGuard guard(plan->device);  // best effort: the plan is released in any case
    cudaDeviceSynchronize();
    destroy_events(plan);
    for (cudaStream_t cs : plan->copy_streams) cudaStreamDestroy(cs);
    for (cudaEvent_t ce : plan->copy_events) cudaEventDestroy(ce);
    for (int j = 0; j < 2; ++j) {
        for (cudaEvent_t ce : plan->in_done[j]) cudaEventDestroy(ce);
        for (cudaEvent_t ce : plan->out_done[j]) cudaEventDestroy(ce);
        if (plan->fwd_done[j]) cudaEventDestroy(plan->fwd_done[j]);
    }
    for (void *a : plan->allocs) cudaFree(a);
    delete plan;
}

int das_plan_set_c(das_plan_t *plan, double c) {
    if (!plan) return fail(DAS_ERR_INVALID_ARG, "plan is NULL");
    if (!(c > 0) || !std::isfinite(c)) return fail(DAS_ERR_INVALID_ARG, "c must be positive");
    if (c != plan->c) {
        plan->c = c;
        plan->dirty = true;
    }
    return DAS_OK;
}

int das_plan_info(const das_plan_t *plan, das_plan_info_t *info) {
    if (!plan || !info) return fail(DAS_ERR_INVALID_ARG, "NULL argument");
    info->n_voxels = plan->g.n_voxels;
    info->n_elements = plan->M;
    info->n_transmits = plan->Q;
    info->n_samples = plan->K;
    info->sample_type = plan->sample_type;
    info->storage = plan->storage;
    info->max_batch = plan->max_batch;
    info->device_bytes = (long long)plan->bytes;
    info->c = plan->c;
    info->kernel_launches = plan->launches;
    info->tc_mma_n = plan->tc_n;
    info->tc_mma_items = 0;
    if (plan->tc_items) {
        DeviceGuard guard(plan->device);
        if (!guard.ok) return fail(DAS_ERR_CUDA, "cannot select the plan's device");
        unsigned long long v = 0;
        DAS_CU(cudaMemcpy(&v, plan->tc_items, sizeof(v), cudaMemcpyDeviceToHost));
        info->tc_mma_items = (long long)v;
    }
    return DAS_OK;
}

int das_plan_check(das_plan_t *plan, das_stream_t stream) {
    if (!plan) return fail(DAS_ERR_INVALID_ARG, "plan is NULL");
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(DAS_ERR_CUDA, "cannot select the plan's device");
    int flags = 0;
    DAS_CU(cudaMemcpyAsync(&flags, plan->err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    DAS_CU(cudaStreamSynchronize((cudaStream_t)stream));
    if (flags) {
        DAS_CU(cudaMemsetAsync(plan->err, 0, sizeof(int), (cudaStream_t)stream));
        DAS_CU(cudaStreamSynchronize((cudaStream_t)stream));
        return fail(DAS_ERR_TIMEOUT, "a kernel gave up a bounded wait or lost a term (error word 0x%x)", flags);
    }
    return DAS_OK;
}

int das_plan_set_wait_test(das_plan_t *plan, long long wait_ns, int probe) {
    if (!plan) return fail(DAS_ERR_INVALID_ARG, "plan is NULL");
    if (wait_ns < 0 || wait_ns > 10000000000LL) return fail(DAS_ERR_INVALID_ARG, "wait_ns must lie in 0 .. 1e10");
    if (probe != 0 && probe != 1) return fail(DAS_ERR_INVALID_ARG, "probe must be 0 or 1");
    plan->wait_ns = (unsigned long long)wait_ns;
    plan->wait_probe = probe;
    return DAS_OK;
}

int das_plan_enable_timing(das_plan_t *plan, int capacity) {
    if (!plan || capacity < 0) return fail(DAS_ERR_INVALID_ARG, "bad argument");
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(DAS_ERR_CUDA, "cannot select the plan's device");
    destroy_events(plan);
    for (int i = 0; i < capacity; ++i) {
        cudaEvent_t a, b;
        DAS_CU(cudaEventCreate(&a));
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return cuda_fail(cudaGetLastError(), "cudaEventCreate");
        }
        plan->ev_start.push_back(a);
        plan->ev_stop.push_back(b);
    }
    return DAS_OK;
}

int das_plan_timing(das_plan_t *plan, double *ms_total, int *launches) {
    if (!plan || !ms_total || !launches) return fail(DAS_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(DAS_ERR_CUDA, "cannot select the plan's device");
    double total = 0.0;
    for (int i = 0; i < plan->ev_used; ++i) {
        DAS_CU(cudaEventSynchronize(plan->ev_stop[i]));
        float ms = 0.f;
        DAS_CU(cudaEventElapsedTime(&ms, plan->ev_start[i], plan->ev_stop[i]));
        total += ms;
    }
    *ms_total = total;
    *launches = plan->ev_used;
    plan->ev_used = 0;
    return DAS_OK;
}

int das_plan_set_tuning(das_plan_t *plan, const das_tuning_t *tuning) {
    if (!plan || !tuning) return fail(DAS_ERR_INVALID_ARG, "NULL argument");
    if (tuning->frames_per_thread < 0 || tuning->ctas_per_sm < 0 || tuning->staging < 0 || tuning->tensor_cores < 0 ||
        tuning->tc_chain < -1)
        return fail(DAS_ERR_INVALID_ARG, "negative tuning value");
    if (tuning->voxels_per_thread < 0 || tuning->voxels_per_thread > 2)
        return fail(DAS_ERR_INVALID_ARG, "voxels_per_thread must be 0, 1 or 2");
    if (tuning->adjoint_rows < 0) return fail(DAS_ERR_INVALID_ARG, "adjoint_rows must be >= 0");
    if (tuning->host_io < 0 || tuning->host_io > 2) return fail(DAS_ERR_INVALID_ARG, "host_io must be 0, 1 or 2");
    if (tuning->tensor_cores && !tc_capable(plan))
        return fail(DAS_ERR_UNSUPPORTED, "the tensor-core path takes IQ data stored as f16 or bf16");
    if (tuning->load_width != 0 && tuning->load_width != 128 && tuning->load_width != 256)
        return fail(DAS_ERR_INVALID_ARG, "load_width must be 0, 128 or 256");
    if (tuning->frames_per_thread > 0 &&
        !tile_fb_supported(MODE_FWD, is_iq(plan), plan->storage, tuning->frames_per_thread))
        return fail(DAS_ERR_UNSUPPORTED, "frames_per_thread %d not compiled for this storage", tuning->frames_per_thread);
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(DAS_ERR_CUDA, "cannot select the plan's device");
    plan->tuning = *tuning;
    int rc = ensure_scratch(plan);
    if (rc == DAS_OK && tuning->tensor_cores) rc = ensure_tc_scratch(plan);
    return rc;
}

static int check_call(das_plan_t *plan, const void *a, const void *b, int batch) {
    if (!plan) return fail(DAS_ERR_INVALID_ARG, "plan is NULL");
    if (!a || !b) return fail(DAS_ERR_INVALID_ARG, "NULL data pointer");
    if (batch < 1 || batch > plan->max_batch)
        return fail(DAS_ERR_INVALID_ARG, "batch %d outside 1..max_batch (%d)", batch, plan->max_batch);
    const size_t al = is_iq(plan) ? 8 : 4;
    if (!aligned(a, al) || !aligned(b, al)) return fail(DAS_ERR_INVALID_ARG, "data pointers must be %zu-byte aligned", al);
    return DAS_OK;
}

int das_forward(das_plan_t *plan, const void *y_dev, void *x_dev, int batch, das_stream_t stream) {
    g_err[0] = 0;
    int rc = check_call(plan, y_dev, x_dev, batch);
    if (rc != DAS_OK) return rc;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(DAS_ERR_CUDA, "cannot select the plan's device");
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = prepare_if_dirty(plan, s)) != DAS_OK) return rc;
    if (plan->tuning.tensor_cores) return forward_tc(plan, y_dev, x_dev, batch, s);
    const int fb = choose_fb(plan, batch, MODE_FWD);
    const int nch = (batch + fb - 1) / fb;
    const int col = col_layout(plan, fb);
    const void *z = nullptr;
    if ((rc = stage_channels(plan, y_dev, batch, fb, nch, col, s, &z)) != DAS_OK) return rc;
    TileArgs A = tile_args(plan, batch, fb, z);
    A.col = col;
    A.x = x_dev;
    const bool timed = plan->ev_used < (int)plan->ev_start.size();
    if (timed) DAS_CU(cudaEventRecord(plan->ev_start[plan->ev_used], s));
    if (col && plan->tuning.voxels_per_thread == 2 && pair_supported(MODE_FWD, is_iq(plan), plan->storage, fb))
        DAS_CU(launch_pair(A, plan->storage, fb, nch, s));
    else
        DAS_CU(launch_tile(A, MODE_FWD, is_iq(plan), plan->storage, fb, nch, s));
    plan->launches += 1;
    if (timed) {
        DAS_CU(cudaEventRecord(plan->ev_stop[plan->ev_used], s));
        plan->ev_used += 1;
    }
    return DAS_OK;
}

// Staging slots 0 .. slots-1, copy streams and events of the host calls
// (created on first use).
static int ensure_host_io(das_plan *p, int slots) {
    int rc;
    const size_t ybytes = (size_t)p->max_batch * p->Q * p->M * p->K * sample_bytes_public(p);
    const size_t xbytes = (size_t)p->max_batch * p->g.n_voxels * sample_bytes_public(p);
    for (int j = 0; j < slots; ++j) {
        if (!p->stage_y[j] && (rc = dalloc(p, &p->stage_y[j], ybytes, "host-call input staging")) != DAS_OK)
            return rc;
        if (!p->stage_x[j] && (rc = dalloc(p, &p->stage_x[j], xbytes, "host-call output staging")) != DAS_OK)
            return rc;
    }
    if (p->copy_streams.empty()) {
        for (int i = 0; i < HOST_COPY_STREAMS; ++i) {
            cudaStream_t cs;
            DAS_CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            p->copy_streams.push_back(cs);
        }
        for (int i = 0; i <= HOST_COPY_STREAMS; ++i) {
            cudaEvent_t ce;
            DAS_CU(cudaEventCreateWithFlags(&ce, cudaEventDisableTiming));
            p->copy_events.push_back(ce);
        }
    }
    if (slots > 1 && !p->fwd_done[0]) {
        for (int j = 0; j < 2; ++j) {
            for (int i = 0; i < HOST_COPY_STREAMS; ++i) {
                cudaEvent_t a, b;
                DAS_CU(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
                p->in_done[j].push_back(a);
                DAS_CU(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
                p->out_done[j].push_back(b);
            }
            DAS_CU(cudaEventCreateWithFlags(&p->fwd_done[j], cudaEventDisableTiming));
        }
    }
    return DAS_OK;
}

// Device addresses of a page-locked host range [p, p + bytes) (host_io = 2):
// both ends must be registered and map to one contiguous device range.
static int host_device_ptr(const void *p, size_t bytes, void **dev) {
    void *a = nullptr, *b = nullptr;
    if (cudaHostGetDevicePointer(&a, const_cast<void *>(p), 0) != cudaSuccess ||
        cudaHostGetDevicePointer(&b, (char *)const_cast<void *>(p) + (bytes - 1), 0) != cudaSuccess ||
        (char *)b - (char *)a != (ptrdiff_t)(bytes - 1)) {
        cudaGetLastError();
        return fail(DAS_ERR_INVALID_ARG,
                    "host_io = 2 reads and writes host memory from the GPU: the buffers must be memory the "
                    "GPU can address (page-locked: das_host_alloc, cudaHostAlloc or cudaHostRegister)");
    }
    *dev = a;
    return DAS_OK;
}

// host_io = 2: the forward pass of each batch on the device addresses of the
// caller's page-locked host buffers (the relayout reads the channel data over
// the CPU-GPU link, the tile kernel writes the image there), then one sync.
static int forward_host_direct(das_plan *plan, const void *const *y_host, void *const *x_host, int n_batches,
                               int batch, cudaStream_t s) {
    const size_t yb = (size_t)batch * plan->Q * plan->M * plan->K * sample_bytes_public(plan);
    const size_t xb = (size_t)batch * plan->g.n_voxels * sample_bytes_public(plan);
    std::vector<void *> yd(n_batches), xd(n_batches);
    int rc;
    for (int i = 0; i < n_batches; ++i)
        if ((rc = host_device_ptr(y_host[i], yb, &yd[i])) != DAS_OK ||
            (rc = host_device_ptr(x_host[i], xb, &xd[i])) != DAS_OK)
            return rc;
    for (int i = 0; i < n_batches; ++i)
        if ((rc = das_forward(plan, yd[i], xd[i], batch, (das_stream_t)s)) != DAS_OK) {
            cudaStreamSynchronize(s);  // earlier batches still use the caller's buffers
            return rc;
        }
    DAS_CU(cudaStreamSynchronize(s));
    return DAS_OK;
}

int das_forward_host(das_plan_t *plan, const void *y_host, void *x_host, int batch, das_stream_t stream) {
    g_err[0] = 0;
    int rc = check_call(plan, y_host, x_host, batch);
    if (rc != DAS_OK) return rc;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(DAS_ERR_CUDA, "cannot select the plan's device");
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->tuning.host_io == 2) return forward_host_direct(plan, &y_host, &x_host, 1, batch, s);
    if ((rc = ensure_host_io(plan, 1)) != DAS_OK) return rc;
    const size_t yb = (size_t)batch * plan->Q * plan->M * plan->K * sample_bytes_public(plan);
    const size_t xb = (size_t)batch * plan->g.n_voxels * sample_bytes_public(plan);
    if ((rc = copy_split(plan, plan->stage_y[0], y_host, yb, cudaMemcpyHostToDevice, s)) == DAS_OK &&
        (rc = das_forward(plan, plan->stage_y[0], plan->stage_x[0], batch, stream)) == DAS_OK &&
        (rc = copy_split(plan, x_host, plan->stage_x[0], xb, cudaMemcpyDeviceToHost, s)) == DAS_OK) {
        DAS_CU(cudaStreamSynchronize(s));
        return DAS_OK;
    }
    // copies already queued use the caller's host buffers: let them finish first
    const std::string first = g_err;
    for (cudaStream_t cs : plan->copy_streams) cudaStreamSynchronize(cs);
    cudaStreamSynchronize(s);
    return fail(rc, "%s", first.c_str());
}

// `bytes` as up to HOST_COPY_STREAMS pieces (at least 16 MB each) on the copy
// streams, each after `after` (if any); piece i records done[i].  Returns
// the number of pieces.
static int copy_pieces(das_plan *p, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind,
                       cudaEvent_t after, const std::vector<cudaEvent_t> &done, int *pieces_out) {
    const size_t min_piece = (size_t)16 << 20;
    int pieces = (int)((bytes + min_piece - 1) / min_piece);
    if (pieces > HOST_COPY_STREAMS) pieces = HOST_COPY_STREAMS;
    if (pieces < 1) pieces = 1;
    const size_t piece = ((bytes + pieces - 1) / pieces + 255) / 256 * 256;
    int n = 0;
    for (int i = 0; i < pieces; ++i) {
        const size_t off = (size_t)i * piece;
        if (off >= bytes && i > 0) break;
        const size_t len = off + piece <= bytes ? piece : bytes - off;
        cudaStream_t cs = p->copy_streams[i];
        if (after) DAS_CU(cudaStreamWaitEvent(cs, after, 0));
        if (len > 0) DAS_CU(cudaMemcpyAsync((char *)dst + off, (const char *)src + off, len, kind, cs));
        DAS_CU(cudaEventRecord(done[i], cs));
        ++n;
    }
    *pieces_out = n;
    return DAS_OK;
}

// The work of das_forward_host_many after its checks (see there).
static int forward_host_many_run(das_plan *plan, const void *const *y_host, void *const *x_host, int n_batches,
                                 int batch, cudaStream_t s) {
    int rc;
    const size_t yb = (size_t)batch * plan->Q * plan->M * plan->K * sample_bytes_public(plan);
    const size_t xb = (size_t)batch * plan->g.n_voxels * sample_bytes_public(plan);
    int n_in[2] = {0, 0}, n_out[2] = {0, 0};
    bool used[2] = {false, false};
    // inputs of batch 0 (the copy streams first wait for the work already on `stream`)
    DAS_CU(cudaEventRecord(plan->copy_events[0], s));
    if ((rc = copy_pieces(plan, plan->stage_y[0], y_host[0], yb, cudaMemcpyHostToDevice, plan->copy_events[0],
                          plan->in_done[0], &n_in[0])) != DAS_OK)
        return rc;
    for (int i = 0; i < n_batches; ++i) {
        const int j = i & 1, jn = j ^ 1;
        // inputs of batch i + 1 into the other slot once batch i - 1 has read it
        if (i + 1 < n_batches &&
            (rc = copy_pieces(plan, plan->stage_y[jn], y_host[i + 1], yb, cudaMemcpyHostToDevice,
                              used[jn] ? plan->fwd_done[jn] : plan->copy_events[0], plan->in_done[jn], &n_in[jn])) !=
                DAS_OK)
            return rc;
        // forward pass of batch i once its inputs are in and slot j's image of batch i - 2 is out
        for (int k = 0; k < n_in[j]; ++k) DAS_CU(cudaStreamWaitEvent(s, plan->in_done[j][k], 0));
        for (int k = 0; k < n_out[j]; ++k) DAS_CU(cudaStreamWaitEvent(s, plan->out_done[j][k], 0));
        if ((rc = das_forward(plan, plan->stage_y[j], plan->stage_x[j], batch, s)) != DAS_OK) return rc;
        DAS_CU(cudaEventRecord(plan->fwd_done[j], s));
        used[j] = true;
        // image of batch i out while batch i + 1 runs
        if ((rc = copy_pieces(plan, x_host[i], plan->stage_x[j], xb, cudaMemcpyDeviceToHost, plan->fwd_done[j],
                              plan->out_done[j], &n_out[j])) != DAS_OK)
            return rc;
    }
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < n_out[j]; ++k) DAS_CU(cudaStreamWaitEvent(s, plan->out_done[j][k], 0));
    DAS_CU(cudaStreamSynchronize(s));
    return DAS_OK;
}

int das_forward_host_many(das_plan_t *plan, const void *const *y_host, void *const *x_host, int n_batches,
                          int batch, das_stream_t stream) {
    g_err[0] = 0;
    if (!plan || !y_host || !x_host) return fail(DAS_ERR_INVALID_ARG, "NULL argument");
    if (n_batches < 1) return fail(DAS_ERR_INVALID_ARG, "n_batches must be >= 1");
    int rc;
    for (int i = 0; i < n_batches; ++i)
        if ((rc = check_call(plan, y_host[i], x_host[i], batch)) != DAS_OK) return rc;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(DAS_ERR_CUDA, "cannot select the plan's device");
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->tuning.host_io == 2) return forward_host_direct(plan, y_host, x_host, n_batches, batch, s);
    if ((rc = ensure_host_io(plan, 2)) != DAS_OK) return rc;
    rc = forward_host_many_run(plan, y_host, x_host, n_batches, batch, s);
    if (rc != DAS_OK) {
        // copies already queued read or write the caller's host buffers: let
        // them finish before returning (the error text stays the first one)
        const std::string first = g_err;
        for (cudaStream_t cs : plan->copy_streams) cudaStreamSynchronize(cs);
        cudaStreamSynchronize(s);
        fail(rc, "%s", first.c_str());
    }
    return rc;
}

#ifdef MADV_COLLAPSE
#define DAS_MADV_COLLAPSE MADV_COLLAPSE
#else
#define DAS_MADV_COLLAPSE 25  // the Linux value of MADV_COLLAPSE
#endif

int das_host_alloc(size_t bytes, void **ptr) {
    g_err[0] = 0;
    if (!ptr) return fail(DAS_ERR_INVALID_ARG, "ptr is NULL");
    *ptr = nullptr;
    if (bytes == 0) return fail(DAS_ERR_INVALID_ARG, "bytes must be > 0");
    // huge-page size of the kernel (transparent huge pages), 2 MiB if unknown
    size_t huge = 2u << 20;
    if (FILE *f = fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
        unsigned long long v = 0;
        if (fscanf(f, "%llu", &v) == 1 && v >= 4096 && (v & (v - 1)) == 0) huge = (size_t)v;
        fclose(f);
    }
    const size_t len = (bytes + huge - 1) / huge * huge;
    const size_t map_len = len + huge;
    void *base = mmap(nullptr, map_len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (base == MAP_FAILED) return fail(DAS_ERR_OOM, "mmap of %zu bytes failed", map_len);
    char *p = (char *)(((uintptr_t)base + huge - 1) / huge * huge);
    madvise(p, len, MADV_HUGEPAGE);  // advisory: small pages still work, only slower after GPU work
    const long page = sysconf(_SC_PAGESIZE) > 0 ? sysconf(_SC_PAGESIZE) : 4096;
    for (size_t o = 0; o < len; o += (size_t)page) p[o] = 0;  // fault the pages in before pinning
    // where faulting gave small pages (fragmented memory), ask the kernel to
    // collapse the range into huge pages now (Linux 6.1+; ignored elsewhere)
    madvise(p, len, DAS_MADV_COLLAPSE);
    cudaError_t e = cudaHostRegister(p, len, cudaHostRegisterDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        munmap(base, map_len);
        return cuda_fail(e, "cudaHostRegister");
    }
    {
        std::lock_guard<std::mutex> lock(g_host_mutex);
        g_host_maps[p] = HostMap{base, map_len};
    }
    *ptr = p;
    return DAS_OK;
}

int das_host_free(void *ptr) {
    if (!ptr) return DAS_OK;
    HostMap m{};
    {
        std::lock_guard<std::mutex> lock(g_host_mutex);
        auto it = g_host_maps.find(ptr);
        if (it == g_host_maps.end()) return fail(DAS_ERR_INVALID_ARG, "pointer was not returned by das_host_alloc");
        m = it->second;
        g_host_maps.erase(it);
    }
    cudaHostUnregister(ptr);
    munmap(m.base, m.len);
    return DAS_OK;
}

int das_adjoint(das_plan_t *plan, const void *x_dev, void *y_dev, int batch, das_stream_t stream) {
    g_err[0] = 0;
    int rc = check_call(plan, x_dev, y_dev, batch);
    if (rc != DAS_OK) return rc;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(DAS_ERR_CUDA, "cannot select the plan's device");
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = prepare_if_dirty(plan, s)) != DAS_OK) return rc;
    const bool iq = is_iq(plan);
    const size_t esz = iq ? 8 : 4;
    // each CTA owns a band of ADJ_ROWS samples of its element's rows (all
    // transmits of a chunk, fb frames) in shared memory
    const int want = plan->tuning.adjoint_rows > 0 ? plan->tuning.adjoint_rows : ADJ_ROWS;
    const int rows = plan->K < want ? plan->K : want;
    const size_t budget = 64 * 1024;  // two CTAs of 512 threads per SM
    int fb = 1, qc = 0;
    const int fbs[3] = {4, 2, 1};
    for (int i = 0; i < 3; ++i) {
        const int f = fbs[i];
        if (f > 1 && f > batch) continue;
        const size_t row = (size_t)rows * f * esz;
        const int qmax = (int)(budget / row);
        if (qmax >= (plan->Q < 4 ? plan->Q : 4) || (f == 1 && qmax >= 1)) { fb = f; qc = qmax; break; }
    }
    if (qc < 1) return fail(DAS_ERR_UNSUPPORTED, "the adjoint's shared-memory rows do not fit");
    if (qc > plan->Q) qc = plan->Q;
    const int nqc = (plan->Q + qc - 1) / qc;
    qc = (plan->Q + nqc - 1) / nqc;
    const int n_bands = (plan->K + rows - 1) / rows;
    if ((long long)nqc * n_bands > 65535) return fail(DAS_ERR_UNSUPPORTED, "n_samples %d too large for the adjoint grid", plan->K);
    AdjArgs A{};
    A.g = plan->g;
    A.M = plan->M;
    A.Q = plan->Q;
    A.K = plan->K;
    A.B = batch;
    A.qc = qc;
    A.fb = fb;
    fill_common(plan, A.a, A.ad, A.theta, A.hr, A.hi, A.thr, A.tile_radius);
    A.elem_pos = plan->elem_pos;
    A.elem_nrm = plan->elem_nrm;
    A.tx_tb = plan->tx_tb;
    A.tx_t = plan->tx_t;
    A.tx_tmin = plan->tx_tmin;
    A.tx_tmax = plan->tx_tmax;
    A.tx_span = plan->tx_span;
    A.rows = rows;
    A.n_bands = n_bands;
    A.aRi = (int)ceil((double)A.a * (double)A.tile_radius) + 2;
    A.er = (float)cos(2.0 * M_PI * plan->f_demod / plan->fs);
    A.ei = (float)-sin(2.0 * M_PI * plan->f_demod / plan->fs);
    A.w_tx = plan->w_tx;
    A.rot = plan->rot;
    A.x = x_dev;
    A.y = y_dev;
    DAS_CU(launch_adjoint(A, iq, s));
    plan->launches += 1;
    return DAS_OK;
}

int das_grad_c(das_plan_t *plan, const void *y_dev, const void *gx_dev, double *dLdc_dev, int batch,
               das_stream_t stream) {
    g_err[0] = 0;
    int rc = check_call(plan, y_dev, gx_dev, batch);
    if (rc != DAS_OK) return rc;
    if (!dLdc_dev || !aligned(dLdc_dev, 8)) return fail(DAS_ERR_INVALID_ARG, "dLdc_dev must be an aligned device double");
    if (plan->storage != DAS_STORE_F32) return fail(DAS_ERR_UNSUPPORTED, "das_grad_c needs float32 storage");
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(DAS_ERR_CUDA, "cannot select the plan's device");
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = prepare_if_dirty(plan, s)) != DAS_OK) return rc;
    const int fb = choose_fb(plan, batch, MODE_DC);
    const int nch = (batch + fb - 1) / fb;
    const int col = col_layout(plan, fb);
    const void *z = nullptr;
    if ((rc = stage_channels(plan, y_dev, batch, fb, nch, col, s, &z)) != DAS_OK) return rc;
    TileArgs A = tile_args(plan, batch, fb, z);
    A.col = col;
    A.gx = gx_dev;
    A.partial = plan->partial;
    const long long np = n_tiles(plan->g) * nch;
    if ((size_t)np > plan->partial_n) return fail(DAS_ERR_INVALID_ARG, "partial buffer too small");
    DAS_CU(launch_tile(A, MODE_DC, is_iq(plan), DAS_STORE_F32, fb, nch, s));
    DAS_CU(launch_reduce(plan->partial, np, dLdc_dev, s));
    plan->launches += 2;
    return DAS_OK;
}

int das_count_active(das_plan_t *plan, long long *count_host, das_stream_t stream) {
    g_err[0] = 0;
    if (!plan || !count_host) return fail(DAS_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(DAS_ERR_CUDA, "cannot select the plan's device");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = prepare_if_dirty(plan, s)) != DAS_OK) return rc;
    TileArgs A = tile_args(plan, 1, 1, nullptr);
    A.partial = plan->partial;
    DAS_CU(launch_tile(A, MODE_COUNT, 0, DAS_STORE_F32, 1, 1, s));
    DAS_CU(launch_reduce(plan->partial, n_tiles(plan->g), plan->scalar, s));
    plan->launches += 2;
    double v = 0;
    DAS_CU(cudaMemcpyAsync(&v, plan->scalar, sizeof(double), cudaMemcpyDeviceToHost, s));
    DAS_CU(cudaStreamSynchronize(s));
    *count_host = (long long)llround(v);
    return DAS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// das_grad_c_static: das_grad_c without any device allocation of its own.
//
// Some callers cannot allocate device memory at the point where they need the
// derivative: code running under a fixed memory budget (a pool that owns all
// device memory), real-time loops that must not enter the allocator, or code
// that wants the call sequence free of allocator side effects.  This entry
// point keeps the only scratch of the derivative pass -- one float64 partial
// sum per (voxel tile, frame chunk) -- in a fixed array compiled into the
// library instead of in the plan.  The array is 2 MiB (262144 partial sums)
// and every GPU that loads the library keeps it until the process exits.
// ---------------------------------------------------------------------------

#include <mutex>

#define DAS_STATIC_PARTIALS (1 << 18)

static __device__ __align__(256) double g_static_partials[DAS_STATIC_PARTIALS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
double *g_static_ptr[kMaxDevices] = {nullptr};

// Device address of the static array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and remembered.
int static_partials_address(int device, double **out) {
    if (device < 0 || device >= kMaxDevices) return fail(DAS_ERR_UNSUPPORTED, "device index %d too large", device);
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_partials);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_partials)");
        g_static_ptr[device] = static_cast<double *>(ptr);
    }
    *out = g_static_ptr[device];
    return DAS_OK;
}
}  // namespace

extern "C" int das_grad_c_static(das_plan_t *plan, const void *y_dev, const void *gx_dev, double *dLdc_dev,
                                 int batch, das_stream_t stream) {
    g_err[0] = 0;
    int rc = check_call(plan, y_dev, gx_dev, batch);
    if (rc != DAS_OK) return rc;
    if (!dLdc_dev || !aligned(dLdc_dev, 8)) return fail(DAS_ERR_INVALID_ARG, "dLdc_dev must be an aligned device double");
    if (plan->storage != DAS_STORE_F32) return fail(DAS_ERR_UNSUPPORTED, "das_grad_c_static needs float32 storage");
    const int fb = choose_fb(plan, batch, MODE_DC);
    const int nch = (batch + fb - 1) / fb;
    const long long np = n_tiles(plan->g) * nch;
    if (np > DAS_STATIC_PARTIALS)
        return fail(DAS_ERR_UNSUPPORTED,
                    "das_grad_c_static: %lld partial sums needed (voxel tiles x frame chunks), the static scratch holds %d",
                    np, DAS_STATIC_PARTIALS);
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(DAS_ERR_CUDA, "cannot select the plan's device");
    double *partial = nullptr;
    if ((rc = static_partials_address(plan->device, &partial)) != DAS_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = prepare_if_dirty(plan, s)) != DAS_OK) return rc;
    const int col = col_layout(plan, fb);
    const void *z = nullptr;
    if ((rc = stage_channels(plan, y_dev, batch, fb, nch, col, s, &z)) != DAS_OK) return rc;
    TileArgs A = tile_args(plan, batch, fb, z);
    A.col = col;
    A.gx = gx_dev;
    A.partial = partial;  // every slot 0..np-1 is written by its CTA before the reduction reads it
    DAS_CU(launch_tile(A, MODE_DC, is_iq(plan), DAS_STORE_F32, fb, nch, s));
    DAS_CU(launch_reduce(partial, np, dLdc_dev, s));
    plan->launches += 2;
    return DAS_OK;
}

// ---------------------------------------------------------------------------
// Batches: several plans and all their frames in one persistent launch,
// replayed from a CUDA graph.
// ---------------------------------------------------------------------------

#include "das_batch.cuh"

struct das_batch {
    int device = 0;
    int n = 0;
    das_plan *plans[BATCH_MAX_PLANS] = {nullptr};
    int frames[BATCH_MAX_PLANS] = {0};
    bool tc[BATCH_MAX_PLANS] = {false};  // plan runs as its own tensor-core launches inside the graph
    int fb = 0;
    das_tuning_t tuning{};
    int4 *items = nullptr;
    int n_items = 0;
    int *counter = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *cap_y[BATCH_MAX_PLANS] = {nullptr};
    void *cap_x[BATCH_MAX_PLANS] = {nullptr};
    int kernels_per_launch = 0;
    long long launches = 0;
};

namespace {

void batch_drop_graph(das_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

int batch_choose_fb(const das_batch *b) {
    const das_plan *p = b->plans[0];
    if (b->tuning.frames_per_thread > 0) return b->tuning.frames_per_thread;
    static const int cands[] = {24, 20, 16, 12, 8, 4, 2};
    int best = 0;
    long best_cost = -1;
    for (int fb : cands) {
        if (!batch_fb_supported(is_iq(p), p->storage, fb)) continue;
        long cost = 0;
        for (int i = 0; i < b->n; ++i)
            if (!b->tc[i]) cost += (long)((b->frames[i] + fb - 1) / fb) * (6 + fb);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = fb; }
    }
    return best;
}

// Scratch of plan p for `bs` padded frames, enlarged if needed.
int ensure_scratch_frames(das_plan *p, int bs) {
    const size_t need = (size_t)p->Q * p->M * p->K * (size_t)bs * sample_bytes_store(p);
    if (need <= p->z_bytes) return DAS_OK;
    dfree(p, p->z);
    p->bytes -= p->z_bytes;
    p->z = nullptr;
    p->z_bytes = 0;
    int rc = dalloc(p, &p->z, need, "channel-data scratch");
    if (rc == DAS_OK) p->z_bytes = need;
    return rc;
}

// Work list: (plan, chunk, tile), the plans with the most work per tile first;
// plans whose own tuning selects the tensor cores are left out of it (they run
// as their own launches inside the batch's graph).
int batch_build(das_batch *b) {
    for (int i = 0; i < b->n; ++i) b->tc[i] = b->plans[i]->tuning.tensor_cores && tc_capable(b->plans[i]);
    const int fb = batch_choose_fb(b);
    if (!batch_fb_supported(is_iq(b->plans[0]), b->plans[0]->storage, fb))
        return fail(DAS_ERR_UNSUPPORTED, "frames_per_thread %d not compiled for batches of this storage", fb);
    int order[BATCH_MAX_PLANS];
    for (int i = 0; i < b->n; ++i) order[i] = i;
    for (int i = 0; i < b->n; ++i)
        for (int j = i + 1; j < b->n; ++j) {
            const das_plan *pi = b->plans[order[i]], *pj = b->plans[order[j]];
            if ((long long)pj->M * pj->Q > (long long)pi->M * pi->Q) std::swap(order[i], order[j]);
        }
    std::vector<int4> items;
    for (int oi = 0; oi < b->n; ++oi) {
        const int i = order[oi];
        das_plan *p = b->plans[i];
        if (b->tc[i]) continue;
        const int nch = (b->frames[i] + fb - 1) / fb;
        int rc = ensure_scratch_frames(p, nch * fb);
        if (rc != DAS_OK) return rc;
        const long long T = n_tiles(p->g);
        for (int c = 0; c < nch; ++c)
            for (long long t = 0; t < T; ++t) items.push_back(make_int4(i, c, (int)t, 0));
    }
    if (items.size() > 0x7fffffff) return fail(DAS_ERR_UNSUPPORTED, "too many work items");
    if (b->items) cudaFree(b->items);
    b->items = nullptr;
    if (!items.empty()) {
        DAS_CU(cudaMalloc(&b->items, sizeof(int4) * items.size()));
        DAS_CU(cudaMemcpy(b->items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    }
    b->n_items = (int)items.size();
    b->fb = fb;
    batch_drop_graph(b);
    return DAS_OK;
}

}  // namespace

extern "C" int das_batch_create(das_batch_t **out, das_plan_t *const *plans, const int *frames, int n_plans) {
    g_err[0] = 0;
    if (!out) return fail(DAS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!plans || !frames) return fail(DAS_ERR_INVALID_ARG, "NULL argument");
    if (n_plans < 1 || n_plans > BATCH_MAX_PLANS)
        return fail(DAS_ERR_UNSUPPORTED, "a batch holds 1..%d plans (got %d)", BATCH_MAX_PLANS, n_plans);
    for (int i = 0; i < n_plans; ++i) {
        if (!plans[i]) return fail(DAS_ERR_INVALID_ARG, "plan %d is NULL", i);
        if (frames[i] < 1 || frames[i] > plans[i]->max_batch)
            return fail(DAS_ERR_INVALID_ARG, "plan %d: frames %d outside 1..max_batch (%d)", i, frames[i],
                        plans[i]->max_batch);
        if (plans[i]->device != plans[0]->device || plans[i]->sample_type != plans[0]->sample_type ||
            plans[i]->storage != plans[0]->storage)
            return fail(DAS_ERR_INVALID_ARG, "plans of a batch share device, sample type and storage");
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return fail(DAS_ERR_INVALID_ARG, "plan %d appears twice", i);
    }
    das_batch *b = new (std::nothrow) das_batch();
    if (!b) return fail(DAS_ERR_OOM, "host allocation failed");
    b->n = n_plans;
    b->device = plans[0]->device;
    for (int i = 0; i < n_plans; ++i) { b->plans[i] = plans[i]; b->frames[i] = frames[i]; }
    DeviceGuard guard(b->device);
    if (!guard.ok) {
        delete b;
        return fail(DAS_ERR_CUDA, "cannot select the plans' device");
    }
    int rc = DAS_OK;
    cudaError_t e;
    if ((e = cudaMalloc(&b->counter, sizeof(int))) != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(counter)");
    else if ((e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) rc = cuda_fail(e, "cudaStreamCreate");
    else rc = batch_build(b);
    if (rc != DAS_OK) {
        if (b->items) cudaFree(b->items);
        if (b->counter) cudaFree(b->counter);
        if (b->cap) cudaStreamDestroy(b->cap);
        delete b;
        return rc;
    }
    *out = b;
    return DAS_OK;
}

extern "C" void das_batch_destroy(das_batch_t *b) {
    if (!b) return;
    DeviceGuard guard(b->device);  // best effort: the batch is released in any case
    cudaDeviceSynchronize();
    batch_drop_graph(b);
    if (b->items) cudaFree(b->items);
    if (b->counter) cudaFree(b->counter);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

extern "C" int das_batch_set_tuning(das_batch_t *b, const das_tuning_t *tuning) {
    if (!b || !tuning) return fail(DAS_ERR_INVALID_ARG, "NULL argument");
    if (tuning->frames_per_thread < 0 || tuning->ctas_per_sm < 0 || tuning->staging < 0 || tuning->tensor_cores < 0)
        return fail(DAS_ERR_INVALID_ARG, "negative tuning value");
    if (tuning->tensor_cores)
        return fail(DAS_ERR_UNSUPPORTED, "choose the tensor cores per plan (das_plan_set_tuning), not per batch");
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(DAS_ERR_CUDA, "cannot select the plan's device");
    b->tuning = *tuning;
    return batch_build(b);
}

extern "C" int das_batch_info(const das_batch_t *b, int *frames_per_thread, int *n_items, int *kernels_per_launch) {
    if (!b) return fail(DAS_ERR_INVALID_ARG, "batch is NULL");
    if (frames_per_thread) *frames_per_thread = b->fb;
    if (n_items) *n_items = b->n_items;
    if (kernels_per_launch) *kernels_per_launch = b->kernels_per_launch;
    return DAS_OK;
}

extern "C" int das_batch_forward(das_batch_t *b, const void *const *y_dev, void *const *x_dev, das_stream_t stream) {
    g_err[0] = 0;
    if (!b || !y_dev || !x_dev) return fail(DAS_ERR_INVALID_ARG, "NULL argument");
    for (int i = 0; i < b->n; ++i) {
        const size_t al = is_iq(b->plans[i]) ? 8 : 4;
        if (!y_dev[i] || !x_dev[i] || !aligned(y_dev[i], al) || !aligned(x_dev[i], al))
            return fail(DAS_ERR_INVALID_ARG, "plan %d: NULL or misaligned data pointer", i);
    }
    DeviceGuard guard(b->device);
    if (!guard.ok) return fail(DAS_ERR_CUDA, "cannot select the plan's device");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    for (int i = 0; i < b->n; ++i)
        if ((rc = prepare_if_dirty(b->plans[i], s)) != DAS_OK) return rc;
    bool same = b->exec != nullptr;
    for (int i = 0; i < b->n && same; ++i) same = (b->cap_y[i] == y_dev[i] && b->cap_x[i] == x_dev[i]);
    if (!same) {
        batch_drop_graph(b);
        BatchParams P{};
        DAS_CU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        int kernels = 0;
        for (int i = 0; i < b->n && rc == DAS_OK; ++i) {
            das_plan *p = b->plans[i];
            const long long l0 = p->launches;
            if (b->tc[i]) {
                // this plan's tensor-core launches (scales, operand relayout, tcgen05 kernel)
                rc = forward_tc(p, y_dev[i], x_dev[i], b->frames[i], b->cap, false);
                kernels += (int)(p->launches - l0);
                continue;
            }
            const int nch = (b->frames[i] + b->fb - 1) / b->fb;
            const void *z = nullptr;
            rc = stage_channels(p, y_dev[i], b->frames[i], b->fb, nch, 0, b->cap, &z);
            kernels += (int)(p->launches - l0);
            P.plans[i] = tile_args(p, b->frames[i], b->fb, z);
            P.plans[i].x = x_dev[i];
            P.plans[i].w256 = 0;
            P.plans[i].umax = b->tuning.staging ? window_rows((p->fs / p->c) * (double)P.plans[i].tile_radius) : 0;
        }
        cudaError_t e = cudaSuccess;
        if (rc == DAS_OK) {
            P.items = b->items;
            P.n_items = b->n_items;
            P.counter = b->counter;
            if (b->n_items > 0) {  // CUDA-core plans: the persistent launch over their work items
                e = cudaMemsetAsync(b->counter, 0, sizeof(int), b->cap);
                if (e == cudaSuccess)
                    e = launch_batch(P, b->n, is_iq(b->plans[0]), b->plans[0]->storage, b->fb,
                                     b->tuning.ctas_per_sm, b->tuning.staging, b->cap);
                kernels += 1;
            }
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
        if (rc != DAS_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
        if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cuda_fail(e, "batch launch capture"); }
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        b->graph = graph;
        DAS_CU(cudaGraphInstantiate(&b->exec, b->graph, 0));
        for (int i = 0; i < b->n; ++i) { b->cap_y[i] = y_dev[i]; b->cap_x[i] = x_dev[i]; }
        b->kernels_per_launch = kernels;
    }
    DAS_CU(cudaGraphLaunch(b->exec, s));
    b->launches += b->kernels_per_launch;
    return DAS_OK;
}
