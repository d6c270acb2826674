/*
 * das_oracle.h -- plain FP64 CPU reference ("oracle") for volumetric
 * delay-and-sum (DAS) beamforming.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this code: only the test-suite, the smoke check and the CPU baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA library under paper_2606_13259_gb300/csrc.
 *
 * What it computes (paper Sec. 2, "Delay-and-sum"):
 *
 *   Eq. 1   tau_qmn = tau^tx_qn + ||p_n - r_m|| / c
 *   Eq. 2   x_bn    = sum_q sum_m  w^tx_qn * w^rx_mn * y_bqm[tau_qmn] * e^{+i 2 pi f_d tau_qmn}
 *
 * with y[tau] the linear interpolation between samples k = floor(tau*fs) and
 * k+1 (Sec. 2, text after Eq. 2).  The readings taken where the paper is
 * silent are spelled out next to each function in das_oracle.c.
 *
 * All arithmetic is IEEE double.  Channel data come in as float32 (the data
 * type the workloads hold) and are widened exactly on read.
 */
#ifndef DAS_ORACLE_H
#define DAS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_TX_DIVERGING = 0, ORACLE_TX_PLANE = 1, ORACLE_TX_NONE = 2 };

typedef struct {
    /* voxel grid: p(ix,iy,iz) = origin + (ix*sx, iy*sy, iz*sz); n = (iz*ny + iy)*nx + ix */
    int nx, ny, nz;
    double origin[3];
    double spacing[3];
    /* receive elements: position and unit direction (normal), [M][3] each */
    int M;
    const double *elem_pos;
    const double *elem_normal;
    /* observations (transmits) */
    int Q;
    const int *tx_kind;     /* ORACLE_TX_* per transmit */
    const double *tx_vec;   /* [Q][3]: virtual source (diverging) or unit propagation direction (plane) */
    const double *w_tx;     /* [Q][N] transmit weight per voxel, or NULL for all ones */
    double t0_ref[3];       /* point at which the transmitted wave defines t = 0 */
    int t0_offset;          /* diverging: 1 subtracts ||v_q - t0_ref|| from the transmit path */
    /* acquisition */
    double c;               /* speed of sound, m/s */
    double fs;              /* sampling rate, Hz */
    double f_demod;         /* demodulation frequency, Hz (0: real RF data) */
    double f_number;        /* receive f-number; <= 0 means the full aperture */
    int K;                  /* samples per channel */
    int iq;                 /* 1: complex (interleaved re,im) channel data; 0: real */
} das_oracle_problem;

/* Forward DAS (Eq. 2).  y: float32 [B][Q][M][K] (complex interleaved when iq).
 * voxels: list of nv voxel indices, or NULL for all N voxels in order.
 * x: double complex interleaved [B][nv]. */
void oracle_forward(const das_oracle_problem *P, const float *y, int B,
                    const long *voxels, long nv, double *x);

/* Same as oracle_forward with a double-precision input y (complex interleaved
 * when iq).  Used by the adjoint identity, which needs FP64 data on both sides. */
void oracle_forward_f64(const das_oracle_problem *P, const double *y, int B,
                        const long *voxels, long nv, double *x);

/* Adjoint DAS^H (the exact conjugate transpose of the linear map in Eq. 2).
 * x: double complex interleaved [B][N].  rows: list of nrows channel rows
 * (index q*M + m), or NULL for all Q*M rows in order.  y: double complex
 * interleaved [B][nrows][K], overwritten. */
void oracle_adjoint(const das_oracle_problem *P, const double *x, int B,
                    const long *rows, long nrows, double *y);

/* Sound-speed derivative: returns Re sum_{b,i} conj(gx_bi) * d x_{b,n_i} / d c
 * over the voxel list (NULL: all N voxels in order), with gx double complex
 * interleaved [B][nv]. */
double oracle_grad_c(const das_oracle_problem *P, const float *y, const double *gx, int B,
                     const long *voxels, long nv);

/* Number of (q, m, n) terms that contribute (inside the receive aperture and
 * with 0 <= k <= K-2). */
long long oracle_count_active(const das_oracle_problem *P);

/* Number of (m, n) pairs whose aperture test lies within rel (relative) of its
 * unshifted threshold without being an exact tie (closer than 1e-9 relative):
 * the pairs whose 0/1 decision could depend on the precision it is taken in. */
long long oracle_count_near_ties(const das_oracle_problem *P, double rel);

/* Number of OpenMP threads the oracle runs with. */
int oracle_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
