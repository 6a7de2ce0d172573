/*
 * pas.h — C ABI of the GB300 (sm_103a) modulated-pyramid single-conjugate AO loop.
 *
 * The calls follow the processing-object chain of the PASSATA paper (Agapito,
 * Puglisi, Esposito, SPIE 2016): atmosphere and propagation, modulated pyramid,
 * CCD, slope computer, modal reconstructor, integrator control and modal DM
 * (Table 1 parameter file, Table 2 main file, Sec. Structure), run once per
 * simulated step by a loop control object (Sec. Build and run a simulation loop).
 * The paper's GPU areas (Sec. GPU acceleration) are the atmosphere propagation,
 * the pyramid propagation and the influence-function multiplication; here every
 * per-step operation of the loop runs in this library's own CUDA kernels.
 *
 * Conventions for every call:
 *   - Device pointers ("d_" prefix) are caller-owned CUDA device memory of the
 *     current device; the library never frees them. Host pointers ("h_" prefix
 *     or documented as host) are read or written synchronously inside the call.
 *   - Arrays are C row-major. Axis 0 of a 2-D map is x (rows), axis 1 is y.
 *   - OPD is in nm, float32. Modal coefficients are nm RMS over the pupil.
 *   - Objects own their internal device buffers, allocated only by *_create and
 *     freed by *_destroy. The per-step calls (advance, measure, apply, update,
 *     loop_step) allocate nothing.
 *   - Every call is asynchronous on the context's stream unless documented
 *     otherwise. Argument errors are returned synchronously as PAS_EINVAL; CUDA
 *     launch errors as PAS_ECUDA; asynchronous device faults surface at the next
 *     call that synchronises. pas_last_error() gives a message per context;
 *     pas_global_error() the message of the last failed create on this thread.
 *   - A NULL handle or pointer where one is required returns PAS_EINVAL.
 */
#ifndef PAS_H
#define PAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PAS_OK = 0,
    PAS_EINVAL = 1,   /* invalid argument or unsupported size */
    PAS_ENOMEM = 2,   /* device allocation failed (no host fallback) */
    PAS_ECUDA = 3,    /* CUDA runtime error */
    PAS_ETIMEOUT = 4, /* a bounded device wait gave up */
    PAS_ESTATE = 5    /* call not valid in the object's current state */
} pas_status;

typedef enum { PAS_FP32 = 0, PAS_BF16 = 1 } pas_precision;

typedef struct pas_ctx_s*   pas_ctx_t;
typedef struct pas_atmo_s*  pas_atmo_t;
typedef struct pas_pyr_s*   pas_pyr_t;
typedef struct pas_recon_s* pas_recon_t;
typedef struct pas_dm_s*    pas_dm_t;
typedef struct pas_loop_s*  pas_loop_t;
typedef struct pas_mlp_s*   pas_mlp_t;
typedef struct pas_batch_s* pas_batch_t;
typedef struct pas_psf_s*   pas_psf_t;
typedef struct pas_sh_s*    pas_sh_t;

/* ------------------------------------------------------------------ context */

/* Library version (major*10000 + minor*100 + patch). Host only, no GPU needed. */
int pas_version(void);

/* Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t, borrowed, may be NULL for the legacy default stream).
 * The context owns nothing else than an error slot and a private stream used
 * only to capture CUDA graphs. */
pas_status pas_ctx_create(void* cuda_stream, pas_ctx_t* out);
void pas_ctx_destroy(pas_ctx_t ctx);
/* Replace the borrowed stream used by later calls. */
pas_status pas_ctx_set_stream(pas_ctx_t ctx, void* cuda_stream);
/* Wait for all work queued on the context stream; returns PAS_ECUDA on a
 * device fault. */
pas_status pas_ctx_synchronize(pas_ctx_t ctx);
const char* pas_last_error(pas_ctx_t ctx);
const char* pas_global_error(void);
/* Host-side fault injection for tests: the n-th following device allocation
 * (n >= 1) made by any *_create fails with PAS_ENOMEM; n = 0 disables. */
void pas_debug_fail_alloc_after(int n);

/* ------------------------------------------------------- pupil geometry (host)
 * Pupil stop (Table 1 pupil_stop, DM.obsratio) and the pupil index data of the
 * slope computer (Table 1 slopec.pupdata_tag; Table 3 calibration). Host-only,
 * integer-exact; no GPU needed.
 *   pixel (i,j) of an Np x Np grid is in the pupil iff
 *     d2 = (2i-Np+1)^2 + (2j-Np+1)^2 <= Np^2  and  d2 >= T,
 *   T = ceil((obs*Np)^2 - 1e-9)  (central obstruction ratio obs).
 *   sub-aperture (r,c) of an n_sub x n_sub grid (b = Np/n_sub pixels a side, Np a
 *   multiple of n_sub) is valid iff 2 * (pupil pixels in its block) >= b^2. */

/* Writes mask[Np*Np] (1 inside, 0 outside) if mask != NULL; *n_pix = count. */
pas_status pas_pupil_mask(int Np, double obs, uint8_t* mask, int32_t* n_pix);
/* Flat indices i*Np+j of the pupil pixels in row-major order into idx[cap]. */
pas_status pas_pupil_pixels(int Np, double obs, int32_t* idx, int32_t cap, int32_t* n_pix);
/* Flat indices r*n_sub+c of the valid sub-apertures in row-major order: twice the
 * pupil area inside the sub-aperture reaches b^2, b = Np / n_sub (not necessarily
 * an integer; exact integer arithmetic on the pixel overlaps). */
pas_status pas_valid_subaps(int Np, double obs, int n_sub, int32_t* valid, int32_t cap,
                            int32_t* n_valid);

/* -------------------------------------------------------------- atmosphere
 * Layered phase screens moved by the wind and summed on the pupil along the
 * on-axis source direction (Table 1 atmo / wind_speed / wind_direction; Table 2
 * get_atmo_container, get_atmo_propagation; Sec. GPU acceleration, "wavefront
 * propagation through phase screens").
 * At step t, pupil pixel (i,j) samples layer l at (i - t*vx[l], j - t*vy[l])
 * (screen pixels, periodic, bilinear; plus the footprint offsets of a view, below). The displacement t*v is one FP64 product
 * from the integer step; floor gives the integer shift and the remainder,
 * rounded to float32, the interpolation weights. */
typedef struct {
    int32_t n_layers;   /* L >= 1 */
    int32_t S;          /* screen side (pixels), >= Np + 2 */
    int32_t Np;         /* pupil side (pixels) */
    const double* vx;   /* host [L]: pixels per step along axis 0 */
    const double* vy;   /* host [L]: pixels per step along axis 1 */
} pas_atmo_params;

/* d_screens: device float32 [L][S][S] OPD in nm (Cn2 weights already applied),
 * caller-owned, must outlive the object. */
pas_status pas_atmo_create(pas_ctx_t ctx, const pas_atmo_params* p, const float* d_screens,
                           pas_atmo_t* out);
/* d_opd: device float32 [Np][Np], the summed OPD of all layers at `step`
 * (every pixel of the square, no pupil mask). */
pas_status pas_atmo_advance(pas_atmo_t atmo, int64_t step, float* d_opd);
/* A second atmosphere object on the same screens and winds, seen along another
 * direction: a natural guide star off axis moves layer l's footprint by h_l theta,
 * so pupil pixel (i,j) samples (i + ox[l] - t vx[l], j + oy[l] - t vy[l]); h_ox,
 * h_oy: host [L] offsets in screen pixels (added to base's own), finite. The view
 * shares base's screens (base's must outlive it); loops and advances use it like
 * any atmosphere. Host only. */
pas_status pas_atmo_create_view(pas_atmo_t base, const double* h_ox, const double* h_oy, pas_atmo_t* out);
/* The same for a source at finite height H (a laser guide star): layer l at height
 * h_l is seen through a footprint shrunk by s_l = 1 - h_l/H about the pupil centre
 * c = (Np - 1)/2 (the cone effect), so pupil pixel (i,j) samples
 * (c + (i - c) s_l + ox[l] - t vx[l], c + (j - c) s_l + oy[l] - t vy[l]), each
 * position one FP64 value per (layer, pixel). h_scale: host [L], each in (0, 1], or
 * NULL (all 1: pas_atmo_create_view). A view of a view composes: the new scale is
 * s_base s and the new offset o_base + s_base o. Host only; EINVAL on a scale
 * outside (0, 1] or a non-finite offset. */
pas_status pas_atmo_create_cone_view(pas_atmo_t base, const double* h_ox, const double* h_oy,
                                     const double* h_scale, pas_atmo_t* out);
/* Tap staging of the loop's residual kernel (Sec. GPU acceleration: the layers are
 * sampled where the pupil pixels see them): for a source at infinity the two screen rows
 * each pupil-row segment of a 64-pixel tile samples are copied by TMA (one-row boxes,
 * from the segment's first column rounded down to 16 bytes, a second box from column 0
 * where the columns wrap around the periodic screen) while the tile's basis streams.
 * pas_atmo_tma: 1 when it applies to this object (S a multiple of 4 and >= 68, screens
 * 16-byte aligned, no cone effect), 0 when the 4-byte asynchronous copies are used, -1
 * for NULL. The values are the same either way, bit for bit. Host only. */
int32_t pas_atmo_tma(pas_atmo_t atmo);
/* Which staging loops created afterwards on this object use: PAS_TAPS_AUTO (default:
 * TMA where pas_atmo_tma is 1 and the DM has a float32 basis of at least 1000 modes,
 * whose stream hides the boxes' latency; the 4-byte copies otherwise), PAS_TAPS_TMA
 * (PAS_EINVAL where pas_atmo_tma is 0), PAS_TAPS_COPY. Views created afterwards
 * inherit it. Host only. */
#define PAS_TAPS_AUTO 0
#define PAS_TAPS_TMA 1
#define PAS_TAPS_COPY 2
pas_status pas_atmo_set_tap_staging(pas_atmo_t atmo, int32_t mode);
/* Tries of the staging's mbarrier wait before it gives up, flags the object and waits
 * again with the long bound (default 2^22, seconds; 0 gives up at once, without
 * testing). Taken by loops created afterwards. Host only. */
pas_status pas_atmo_set_wait_limit(pas_atmo_t atmo, uint32_t tries);
/* Synchronous: PAS_ETIMEOUT if a staging wait of a residual on this atmosphere (or a
 * view of it) gave up since the last check (the flag is cleared); h_fault optional:
 * bit 0 a first wait gave up, bit 1 the second too. */
pas_status pas_atmo_check(pas_atmo_t atmo, uint32_t* h_fault);
void pas_atmo_destroy(pas_atmo_t atmo);

/* ------------------------------------------------------ modulated pyramid
 * Modulated four-face pyramid wavefront sensor, CCD binning and slope computer
 * (Table 1 pyramid, detector, slopec; Sec. GPU acceleration, "pyramid
 * propagation from wavefront to detector plane").
 * For each modulation point k (theta_k = 2 pi k / K from axis 0, radius
 * mod_radius lambda/D) the pupil field A exp(i(2 pi opd/lambda + psi_k)) is
 * centred in an N x N grid, taken to the focal plane by the centred unitary DFT,
 * multiplied by exp(i 2 pi delta (|u~|+|v~|)/N) and brought back; the intensity
 * averaged over k is summed into b x b detector pixels, b = N/(2 n_sub).
 * Slopes over the valid sub-apertures j (detector quadrants q_ab, a = row half,
 * b = column half, sub-aperture (r,c) at pixel (a*n_sub+r, b*n_sub+c)):
 *   Sx = (q10+q11-q00-q01)/F,  Sy = (q01+q11-q00-q10)/F,
 *   F = mean over valid j of (q00+q01+q10+q11); output [Sx(0..nv-1), Sy(..)] - sn.
 * Requirements: N = 2*Np, delta = N/4, N a multiple of 2*n_sub, N in the
 * supported set (see pas_pyr_supported), K even or odd >= 1. */
typedef struct {
    int32_t Np;            /* pupil pixels across */
    int32_t N;             /* FFT grid side */
    int32_t K;             /* modulation points */
    int32_t n_sub;         /* sub-apertures across */
    double mod_radius;     /* lambda/D */
    double wavelength_nm;  /* sensing wavelength */
    double obs;            /* central obstruction ratio */
    int32_t local_norm;    /* 0: global flux normalisation, 1: per sub-aperture */
} pas_pyr_params;

/* 1 if the FFT size N has compiled kernels, else 0. Host only. */
int pas_pyr_supported(int N);
/* h_valid: host int32 [n_valid] flat sub-aperture indices (ascending), or NULL
 * to use the geometric rule above. The object starts with a zero slope
 * reference and noise off. */
pas_status pas_pyr_create(pas_ctx_t ctx, const pas_pyr_params* p, const int32_t* h_valid,
                          int32_t n_valid, pas_pyr_t* out);
/* The same sensor looking at an extended incoherent source (Sec. History/Reference
 * works: extended, non point-like, reference sources; Sec. Conclusions: the costly
 * case at ELT scale): n_points >= 1 point sources at offsets (h_ex[q], h_ey[q])
 * lambda/D from the source centre along axes 0 and 1 (the modulation radius's unit
 * and sign: a point at (r, 0) tilts the wavefront like the modulation point at
 * theta = 0), with relative intensities h_w[q] >= 0 (normalised to sum 1; NULL:
 * equal). Every measurement is sum_q w_q I_q, I_q the modulated intensity of point
 * q: K n_points FFT pairs, each point q riding on the modulation circle at
 * (R cos theta_k + ex_q, R sin theta_k + ey_q); points of equal ey and equal
 * sin theta share one rows pass, and w_q enters as the amplitude sqrt(w_q n_points)
 * of the point's column tilt. Requires K n_points <= 4096. Everything else is
 * pas_pyr_create's (reference slopes, noise, measurement, loops). EINVAL on
 * non-finite offsets, negative or all-zero weights. */
pas_status pas_pyr_create_extended(pas_ctx_t ctx, const pas_pyr_params* p, const int32_t* h_valid,
                                   int32_t n_valid, const double* h_ex, const double* h_ey,
                                   const double* h_w, int32_t n_points, pas_pyr_t* out);
int32_t pas_pyr_n_valid(pas_pyr_t pyr);
/* Copy the valid sub-aperture list to host memory (synchronous). */
pas_status pas_pyr_get_valid(pas_pyr_t pyr, int32_t* h_valid, int32_t cap);
/* d_sn: device float32 [2*n_valid] slope reference (copied), NULL = zero. */
pas_status pas_pyr_set_reference(pas_pyr_t pyr, const float* d_sn);
/* Detector noise (Table 1 detector: photon_noise, readout_noise, readout_level):
 * photons_per_frame <= 0 disables photon noise and keeps the frame in intensity
 * units. With photons > 0 the frame is in photo-electrons:
 *   pix_p = Poisson(photons * I_p / n_pupil_pixels) + read_noise_e * N(0,1),
 * drawn from Philox-4x32-10 (key = seed, counter = (p, frame, block)).
 * `frame_index` sets the counter of the next frame; each measure increments it. */
pas_status pas_pyr_set_noise(pas_pyr_t pyr, double photons_per_frame, double read_noise_e,
                             uint64_t seed, int64_t frame_index);
/* d_opd: device float32 [Np][Np] residual OPD (values outside the pupil are
 * ignored). d_frame: device float32 [2n_sub][2n_sub] out (may be NULL).
 * d_slopes: device float32 [2*n_valid] out (may be NULL). */
pas_status pas_pyr_measure(pas_pyr_t pyr, const float* d_opd, float* d_frame, float* d_slopes);
/* Allocation-free pyramid measurement (the paper has no counterpart).
 * For callers that may not allocate device memory once they run (an application
 * whose allocator forbids cudaMalloc after start-up, code running while another
 * library owns the device allocator, a moment when an allocation would stall the
 * device): it computes what pas_pyr_create + pas_pyr_measure compute (noiseless,
 * default launch geometry) without creating an object and without allocating.
 * Its intermediates live in one array of PAS_STATIC_SCRATCH_BYTES of device memory
 * compiled into this library, held by every GPU that loads it until the process
 * exits. Geometries that need more (e.g. N = 960 with 32 modulation points) are
 * rejected with PAS_EINVAL and a message giving the bytes needed; also N <= 960,
 * K <= 256, n_sub <= 128.
 *   p: as for pas_pyr_create; h_valid (host, ascending) / n_valid or NULL for the
 *   geometric rule; d_sn: device [2 n_valid] slope reference or NULL;
 *   d_opd: device [Np][Np] input; d_frame: device [2n_sub]^2 output (required);
 *   d_slopes: device [2 n_valid] output or NULL; cuda_stream: cudaStream_t or NULL.
 * The first call on a device (with that device current) looks up the array's
 * device address once; make that first call before any stream capture. Every call
 * uses the same array and leaves its contents behind: the call clears what has to
 * start at zero itself, and calls whose work overlaps on the GPU (other streams,
 * other threads) race on it. Its small tables (twiddles, mask, tilts, valid map)
 * are built in host arrays of the library, under a lock held until they have been
 * copied onto the stream (concurrent host calls take turns; nothing large goes on
 * the caller's stack). Because those copies read host memory that the next call
 * reuses, a call on a stream that is being captured is refused with PAS_EINVAL
 * before anything is enqueued. */
#define PAS_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)
pas_status pas_pyr_measure_static(const pas_pyr_params* p, const int32_t* h_valid, int32_t n_valid,
                                  const float* d_sn, const float* d_opd, float* d_frame,
                                  float* d_slopes, void* cuda_stream);
/* Stand-alone detector noise on a frame (same rule as above; frame counter
 * given explicitly; in-place allowed). n = number of pixels. */
pas_status pas_ccd_noise(pas_ctx_t ctx, const float* d_in, float* d_out, int32_t n,
                         double photons_per_frame, int32_t n_pupil_pixels,
                         double read_noise_e, uint64_t seed, int64_t frame_index);
void pas_pyr_destroy(pas_pyr_t pyr);

/* Launch geometry of the pyramid kernels: rows pass = pupil rows per CTA and the
 * number of chunks the distinct sin(theta_k) values are split into (the OPD
 * phasor of a row is computed once per chunk); columns pass = number of groups
 * of modulation points (each CTA accumulates |g|^2 over its group) and the
 * number of CTAs sharing one detector column's b = N / (2 n_sub) fine columns
 * (smaller CTAs, more of them resident per SM). */
typedef struct {
    int32_t rows_per_cta;   /* 1, 2, 4, 8, or 16 where that CTA's shared memory fits */
    int32_t row_chunks;     /* 1 .. number of distinct sin(theta_k) */
    int32_t col_groups;     /* 1 .. K */
    int32_t col_split;      /* 1, or a divisor <= 8 of b when b is an integer */
} pas_pyr_tuning;
pas_status pas_pyr_get_tuning(pas_pyr_t pyr, pas_pyr_tuning* h_out);
/* Values are rounded to the nearest realisable split; results do not depend on
 * the geometry beyond float32 summation order of the modulation groups. */
pas_status pas_pyr_set_tuning(pas_pyr_t pyr, const pas_pyr_tuning* h_t);
/* Autotuner: times each candidate geometry (rows_per_cta 2/4/8/16 x every chunk
 * count; every column group count x every column split) with CUDA events over
 * `iters` launches on d_opd (device [Np][Np]), keeps the fastest and writes it
 * to h_out (may be NULL). Synchronous; overwrites the object's internal frame; do not call while
 * the context stream is being captured. */
pas_status pas_pyr_autotune(pas_pyr_t pyr, const float* d_opd, int32_t iters, pas_pyr_tuning* h_out);

/* ------------------------------------------------- modal reconstructor
 * Modal reconstructor (Table 1 modalrec.recmat_tag): dmodes = R * slopes.
 * h_R: host float32 [n_modes][n_slopes] row-major, copied. PAS_BF16 stores R in
 * bfloat16 with one float32 scale per row (row max |R|) and accumulates in
 * float32. */
pas_status pas_recon_create(pas_ctx_t ctx, const float* h_R, int32_t n_modes, int32_t n_slopes,
                            pas_precision prec, pas_recon_t* out);
/* d_slopes: device float32 [n_slopes]; d_dmodes: device float32 [n_modes] out. */
pas_status pas_recon_apply(pas_recon_t rec, const float* d_slopes, float* d_dmodes);
/* Synchronous check of the reconstructor's bounded waits (long slope vectors stream
 * R through bulk copies whose waits give up after a bound): PAS_ETIMEOUT if one gave
 * up since the last check (the flag is then cleared); h_fault (optional) receives
 * the flag bits. */
pas_status pas_recon_check(pas_recon_t rec, uint32_t* h_fault);
void pas_recon_destroy(pas_recon_t rec);

/* ------------------------------------------------------------- modal DM
 * Integrator control and modal DM (Table 1 control: type 'INT', int_gain;
 * Table 1 DM; Sec. GPU acceleration, "influence function multiplication").
 * h_M: host float32 [n_pix][n_modes] modal basis over the pupil pixels listed
 * (row-major order) by pas_pupil_pixels(Np, obs); copied (stored mode-major).
 * prec: PAS_FP32 keeps the basis in float32; PAS_BF16 rounds it to bfloat16
 * (nearest even; half the bytes the residual streams every step). Products and
 * sums are float32 in both cases. */
pas_status pas_dm_create(pas_ctx_t ctx, const float* h_M, int32_t n_pix, int32_t n_modes,
                         int32_t Np, double obs, pas_precision prec, pas_dm_t* out);
/* Integrator then DM shape:
 *   if d_dmodes != NULL:  cmd[m] += gain[m] * dmodes[m]   (d_gain NULL: gain 1)
 *   if d_opd_dm != NULL:  opd_dm = M * cmd on the pupil pixels, 0 elsewhere
 * d_cmd: device float32 [n_modes] in/out; d_opd_dm: device float32 [Np][Np]. */
pas_status pas_dm_update(pas_dm_t dm, const float* d_dmodes, const float* d_gain, float* d_cmd,
                         float* d_opd_dm);
/* Residual seen by the sensor: opd_res = mask * (opd_atm - M * cmd).
 * d_opd_atm, d_opd_res: device float32 [Np][Np] (may alias); d_cmd [n_modes]. */
pas_status pas_dm_residual(pas_dm_t dm, const float* d_opd_atm, const float* d_cmd,
                           float* d_opd_res);
/* Modal projection (modal analysis of an OPD on the DM basis):
 * coeffs = (1/n_pix) M^T opd over the pupil pixels, the least-squares
 * coefficients when M^T M = n_pix I (orthonormalised basis, nm RMS).
 * d_opd: device float32 [Np][Np]; d_coeffs: device float32 [n_modes] out. */
pas_status pas_dm_project(pas_dm_t dm, const float* d_opd, float* d_coeffs);
void pas_dm_destroy(pas_dm_t dm);

/* ------------------------------------------------------------------ loop
 * Loop control (Sec. Structure; Table 2 loop.add / loop.run): one step runs
 *   atmosphere -> residual (DM command of step t-delay) -> pyramid -> CCD ->
 *   slopes -> reconstructor -> integrator
 * on the context stream. The first call captures one step as a CUDA graph (on
 * the context's private stream) and later calls replay it; call it before
 * capturing anything else on the same stream. The integrator state, the
 * step counter and the per-step residual WFE live on the device. */
typedef struct {
    int64_t step;        /* steps completed */
    double wfe_nm;       /* residual WFE (piston removed) of the last step */
} pas_loop_stats;

/* d_gain: device float32 [n_modes] per-mode integrator gain (copied).
 * delay >= 1: the measurement at step t sees the command of step t - delay.
 * wfe_history: number of per-step WFE values kept (ring buffer, >= 1). */
pas_status pas_loop_create(pas_ctx_t ctx, pas_atmo_t atmo, pas_pyr_t pyr, pas_recon_t rec,
                           pas_dm_t dm, const float* d_gain, int32_t delay,
                           int32_t wfe_history, pas_loop_t* out);
/* The same loop with a Shack-Hartmann sensor (pas_sh_*) in place of the pyramid:
 * a step is residual -> lenslet spots (with the sensor's detector noise, the step
 * as frame index) and centroid slopes -> reconstructor and integrator (the frame of
 * pas_loop_buffers is the sensor's). Everything
 * else (steps, state, buffers, learned reconstructor, batches) works the same;
 * pas_loop_profile answers PAS_ESTATE (its kernel list is the pyramid loop's). */
pas_status pas_loop_create_sh(pas_ctx_t ctx, pas_atmo_t atmo, pas_sh_t sh, pas_recon_t rec,
                              pas_dm_t dm, const float* d_gain, int32_t delay,
                              int32_t wfe_history, pas_loop_t* out);
/* Run n_steps >= 0 steps. If h_stats != NULL the call synchronises and fills it. */
pas_status pas_loop_step(pas_loop_t loop, int32_t n_steps, pas_loop_stats* h_stats);
/* Same step launched kernel by kernel without the graph (for comparison). */
pas_status pas_loop_step_eager(pas_loop_t loop, int32_t n_steps);
/* Device views of the loop's buffers (owned by the loop; valid until destroy):
 * opd_res [Np][Np], frame [2n_sub]^2, slopes [2nv], dmodes [n_modes],
 * cmd [n_modes] (command of the last completed step), wfe [wfe_history]
 * (float64, entry t mod history = WFE of step t). Any pointer may be NULL. */
pas_status pas_loop_buffers(pas_loop_t loop, float** opd_res, float** frame, float** slopes,
                            float** dmodes, float** cmd, double** wfe);
/* Checkpoint / resume: the state is the step counter, the integrator ring
 * (delay x n_modes float32) and the noise frame counter; h_cmd_ring may be NULL
 * on get to query only the step. Synchronous. */
pas_status pas_loop_get_state(pas_loop_t loop, int64_t* step, float* h_cmd_ring);
pas_status pas_loop_set_state(pas_loop_t loop, int64_t step, const float* h_cmd_ring);
/* A detector integrating n_int >= 1 simulation steps per frame (Sec. Structure: a
 * CCD integrating its input for several steps, the objects using its frames
 * following its lower rate): the sensor's (pyramid or Shack-Hartmann) noiseless
 * frames of the steps add up and
 * are read out at each step t with (t + 1) mod n_int = 0 as the window's mean
 * (windows aligned to the step counter), then noise, slopes, reconstruction and
 * integrator run; at the other steps the slopes keep their value and the command
 * is held (the delay still counts steps). n_int = 1 restores one frame per step.
 * The accumulator starts empty (also after pas_loop_set_state). The next step
 * captures a new graph. PAS_ESTATE for a loop with a learned reconstructor;
 * PAS_EINVAL outside 1 .. 2^20. Synchronous. */
pas_status pas_loop_set_integration(pas_loop_t loop, int32_t n_int);
void pas_loop_destroy(pas_loop_t loop);

/* Profiling: run n_steps >= 1 steps, each one launch of a CUDA graph of the step
 * with event-record nodes between its kernels (GPU-side timing, no host launch
 * gaps), synchronising after each, and write the mean duration in ms of each
 * kernel into h_ms[0 .. *n_kernels-1] (cap >= PAS_LOOP_KERNELS). The steps advance
 * the loop like pas_loop_step.
 * The step's kernels, in order: residual (wind-shifted layers sampled at the
 * pupil pixels, - DM shape), pyramid rows pass, pyramid columns pass (+ detector
 * frame and noise in the last CTA of each detector column), slopes, reconstructor + integrator (+ step counter);
 * with a learned reconstructor attached the last entry spans its layer kernels. */
#define PAS_LOOP_KERNELS 5
pas_status pas_loop_profile(pas_loop_t loop, int32_t n_steps, float* h_ms, int32_t cap,
                            int32_t* n_kernels);
/* A PSF camera inside the loop's step graph (Table 2: loop.add(psf); Table 1 camera): from
 * step start_step on, every step's PSF of the loop's residual OPD (the sensing direction) is
 * added to d_psf (device float32 [N][N], N = pas_psf_size) and its Strehl ratio written to
 * d_sr[t mod sr_len] (device float64, or NULL) for step t. The camera's two passes run on a
 * stream of the loop's own after the residual kernel, beside the sensor, and join before the
 * reconstruction. psf = NULL detaches. The camera's pupil must be the loop's (PAS_EINVAL);
 * buffers are borrowed and must outlive the attachment. Synchronises the context stream;
 * the step graph is captured again at the next step. Persistent batches refuse loops with
 * a camera; graph-branch batches step it with the loop. */
pas_status pas_loop_attach_camera(pas_loop_t loop, pas_psf_t psf, float* d_psf, double* d_sr, int32_t sr_len,
                                  int64_t start_step);
/* Name of kernel `idx` of pas_loop_profile (static string), NULL if out of range. */
const char* pas_loop_kernel_name(int32_t idx);

/* ----------------------------------------------------------------- batches
 * Many independent loops (Monte-Carlo realisations, of equal or different
 * sizes) stepped by one CUDA-graph launch per step: the graph holds every loop's
 * step as a parallel branch (the paper runs its Monte-Carlo cases as separate
 * simulations; this is the GPU-side batching of them). The loops keep their own
 * state, buffers and statistics (pas_loop_step(loop, 0, &stats) reads them) and
 * must not be stepped or destroyed while the batch exists; re-configuring one
 * (pas_loop_set_mlp, pas_loop_set_integration, pas_loop_attach_camera) returns PAS_ESTATE
 * until every batch holding it is destroyed. Creation synchronises every loop's stream and captures the graph
 * on `ctx`'s private stream; steps run on `ctx`'s stream. Two loops of a batch may
 * share atmosphere, DM and reconstructor objects but not a sensor object (PAS_EINVAL).
 * Loops that share one DM object (realisations of one system) and whose sources are at
 * infinity get their residuals from one pass over the basis per step: the commands of
 * the group are gathered, then each CTA streams one tile of the basis once for up to
 * 8 (bf16 basis: 4) loops; each loop's residual and WFE equal those of its own
 * residual kernel, bit for bit (pas_batch_n_residual_groups). */
pas_status pas_batch_create(pas_ctx_t ctx, pas_loop_t* loops, int32_t n_loops, pas_batch_t* out);
/* pas_batch_create with flags. PAS_BATCH_PERSISTENT: the pyramid loops' rows and
 * columns passes run as one persistent launch per transform length instead of two
 * launches per loop. Its CTAs (as many as the SMs hold) draw tasks from one queue:
 * every loop's rows-pass tasks (a group of pupil rows x a chunk of the sin values),
 * then every loop's columns-pass tasks (a detector column x a group of modulation
 * points x a column part), each task one CTA of the loop's own launches, so every
 * frame, slope and command equals that of the loop stepped alone, bit for bit. A
 * columns task starts once its loop's rows pass is complete; that wait is bounded
 * (pas_batch_set_wait_limit): when it runs out the task transforms nothing, the
 * launch still completes and pas_batch_check returns PAS_ETIMEOUT. The residuals run
 * first (one kernel per loop), the slopes and reconstructions after the launch;
 * Shack-Hartmann loops are stepped whole beside it. */
#define PAS_BATCH_PERSISTENT 1u
pas_status pas_batch_create_ex(pas_ctx_t ctx, pas_loop_t* loops, int32_t n_loops, uint32_t flags,
                               pas_batch_t* out);
/* n_steps >= 0 steps of every loop of the batch, asynchronous. */
pas_status pas_batch_step(pas_batch_t batch, int32_t n_steps);
/* Number of loops, -1 for a NULL handle. Host only. */
int32_t pas_batch_size(pas_batch_t batch);
/* Loops of the batch that share one PAS_BF16 reconstructor object (one frame per step,
 * no network) are reconstructed together: their slopes, as bf16, form the columns of S,
 * and one tensor-core product C = R S^T (float32 accumulation) gives every loop's
 * modal update, the integrator applied per loop in the product's epilogue (R is read
 * once per step instead of once per loop). Groups of up to 128 loops, in loop order.
 * Loops that share one network (pas_loop_set_mlp) form one group likewise: one batched
 * forward of their slopes through the tensor-core layers per step (bf16 inputs and
 * activations, float32 accumulation), then each loop's integrator on its output; more
 * loops sharing a network than min(128, its batch size) is PAS_EINVAL (the network keeps
 * one set of intermediates).
 * pas_batch_n_groups: how many such groups; pas_batch_kernels_per_step: kernels one
 * step launches; pas_batch_check: synchronous, PAS_ETIMEOUT if a product's bounded
 * wait gave up since the last check (h_fault optional: the flag bits). */
int32_t pas_batch_n_groups(pas_batch_t batch);
int32_t pas_batch_kernels_per_step(pas_batch_t batch);
/* h_fault bit 8 (0x100): a persistent launch's wait gave up; PAS_ETIMEOUT then too. */
pas_status pas_batch_check(pas_batch_t batch, uint32_t* h_fault);
/* Persistent launches per step (one per transform length), 0 for a batch created
 * without PAS_BATCH_PERSISTENT, -1 for a NULL handle. Host only. */
int32_t pas_batch_n_persistent(pas_batch_t batch);
/* Geometry of persistent launch g (0 <= g < pas_batch_n_persistent), h_geo[8]: transform
 * length N, CTAs, threads per CTA, dynamic shared bytes per CTA, pupil rows per rows
 * task, sin values per rows task (at most), rows tasks, columns tasks. The columns tasks
 * keep each loop's own geometry; the rows tasks' geometry (which does not change the
 * result) is chosen for the launch's CTA. Host only. */
pas_status pas_batch_persistent_geometry(pas_batch_t batch, int32_t g, int32_t* h_geo);
/* Groups of loops sharing a DM object whose residuals are computed together; -1 for a
 * NULL handle. Host only. */
int32_t pas_batch_n_residual_groups(pas_batch_t batch);
/* Polls (about 0.3 us each) a columns task makes for its loop's rows pass before it
 * gives up; default 2^21 (about a second). Synchronises `ctx`'s stream. PAS_EINVAL for
 * a batch without persistent launches or a negative limit. */
pas_status pas_batch_set_wait_limit(pas_batch_t batch, int64_t polls);
/* Diagnostic of those waits: one persistent launch with the rows pass withheld, so that
 * every columns task waits for a count nothing advances, gives up after the wait limit
 * and transforms nothing. Synchronous; returns what pas_batch_check returns after it
 * (PAS_ETIMEOUT, h_fault bit 8). The loops' frames and slopes buffers, and the
 * accumulated frame of an integrating detector, are left undefined; their step counters,
 * commands and statistics are untouched. */
pas_status pas_batch_probe_waits(pas_batch_t batch, uint32_t* h_fault);
void pas_batch_destroy(pas_batch_t batch);

/* -------------------------------------------------------------- PSF camera
 * Point-spread function and Strehl ratio of the residual field (Table 1 camera:
 * wavelengthInNm, nd = "padding coefficient for PSF computation"; Table 2
 * psf.in_ef, psf.out_sr, psf.out_int_psf; Sec. GPU acceleration, "PSF generation
 * from residual wavefront"). E = A exp(2 pi i opd / lambda) on the Np x Np pupil
 * (A = pas_pupil_mask), zero-padded to N = nd Np;
 *   PSF(p, q) = |sum_ij E(i,j) exp(-2 pi i ((p - N/2) i + (q - N/2) j) / N)|^2 / (sum A)^2,
 * so the zero frequency sits at (N/2, N/2), a diffraction-limited pupil peaks at 1
 * there and one pixel is lambda / (nd D). The Strehl ratio is the PSF value at
 * (N/2, N/2) = |sum A exp(i phi)|^2 / (sum A)^2. The integrated PSF is the sum of
 * the per-step PSFs from a start step on (accumulate = 1 from that step).
 * Supported pupils Np = 48, 64, 120, 128, 240, 256, 480 and padding 1 <= nd <= 16
 * (PAS_EINVAL otherwise). The object owns its tables and an N x Np complex
 * intermediate. */
pas_status pas_psf_create(pas_ctx_t ctx, int32_t Np, int32_t nd, double wavelength_nm, double obs,
                          pas_psf_t* out);
/* N = nd Np, or -1 for a NULL handle. Host only. */
int32_t pas_psf_size(pas_psf_t psf);
/* d_opd: device float32 [Np][Np] residual OPD in nm (values outside the pupil are
 * ignored); d_psf: device float32 [N][N], written (accumulate = 0) or added to
 * (accumulate = 1); d_strehl: device float64 scalar or NULL, the Strehl ratio.
 * Asynchronous on the context stream; allocates nothing (graph-capturable). */
pas_status pas_psf_compute(pas_psf_t psf, const float* d_opd, float* d_psf, int32_t accumulate,
                           double* d_strehl);
void pas_psf_destroy(pas_psf_t psf);

/* ------------------------------------------------------ Shack-Hartmann WFS
 * The framework's second sensor type (Sec. GPU acceleration, "Pyramid and Shack
 * Hartmann propagation (from wavefront to detector plane)"; the paper gives no
 * parameters). An n_sub x n_sub lenslet array on the Np x Np pupil, b = Np / n_sub
 * pupil pixels per lenslet (integer); lenslet (r, c)'s field E = A exp(2 pi i opd /
 * lambda) zero-padded to M x M, M = ovs b (even, <= 32), gives the spot
 *   I(k, l) = |sum_ij E(i, j) exp(-2 pi i ((k - M/2) i + (l - M/2) j) / M)|^2 / M^2
 * (zero frequency at pixel (M/2, M/2); one pixel = lambda / (ovs d); a spot sums to
 * its lenslet's lit pupil pixels). Spots tile the frame [(n_sub M)][(n_sub M)], lenslet
 * (r, c) at rows r M .. r M + M - 1, columns c M .. c M + M - 1. Slopes: centre of
 * gravity about (M/2, M/2) in pixels, x along axis 0, layout [x; y] over the valid
 * lenslets (ascending r n_sub + c; NULL h_valid: the pyramid's geometric rule, see
 * pas_valid_subaps), minus the reference (pas_sh_set_reference). */
pas_status pas_sh_create(pas_ctx_t ctx, int32_t Np, int32_t n_sub, int32_t ovs, double wavelength_nm,
                         double obs, const int32_t* h_valid, int32_t n_valid, pas_sh_t* out);
/* Number of valid lenslets; side of the frame (n_sub M); -1 for a NULL handle. Host only. */
int32_t pas_sh_n_valid(pas_sh_t sh);
int32_t pas_sh_frame_side(pas_sh_t sh);
/* Copy the valid lenslet indices to host memory (cap >= n_valid). Synchronous. */
pas_status pas_sh_get_valid(pas_sh_t sh, int32_t* h_valid, int32_t cap);
/* d_ref: device float32 [2 n_valid] reference slopes (copied), NULL to clear. */
pas_status pas_sh_set_reference(pas_sh_t sh, const float* d_ref);
/* Detector noise on the frame, as pas_pyr_set_noise: photons_per_frame <= 0 keeps the
 * frame in intensity units (no noise); otherwise pix_p = Poisson(photons * I_p /
 * n_pupil_pixels) + read_noise_e * N(0,1) from Philox-4x32-10 (key = seed, counter =
 * (p, frame, block), p the frame pixel), and the slopes are the noisy frame's
 * centroids. `frame_index` is the counter of the next standalone measurement (each
 * increments it); in a loop the loop's step is the frame index. Synchronous. */
pas_status pas_sh_set_noise(pas_sh_t sh, double photons_per_frame, double read_noise_e,
                            uint64_t seed, int64_t frame_index);
/* d_opd: device float32 [Np][Np] (nm); d_frame (may be NULL): device float32
 * [(n_sub M)^2]; d_slopes (may be NULL): device float32 [2 n_valid]. Asynchronous on
 * the context stream; allocates nothing. */
pas_status pas_sh_measure(pas_sh_t sh, const float* d_opd, float* d_frame, float* d_slopes);
void pas_sh_destroy(pas_sh_t sh);

/* -------------------------------------------------- learned reconstructor
 * A multilayer perceptron from slopes to modal coefficients, used by the loop
 * in place of the linear modal reconstructor (Table 1 modalrec). The paper's
 * reconstructor is linear; this network is an extension of it:
 *   x = (s - mean) * inv_std                      (per slope, set by set_norm)
 *   h_l = gelu(W_l h_{l-1} + b_l), l < L - 1      gelu(z) = z * Phi(z) (erf form)
 *   out = W_{L-1} h_{L-2} + b_{L-1}
 * trained on the mean squared error mean_{b,o} (out - y)^2 with Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 * Parameters travel as one packed float32 vector: W_0 ([sizes[1]][sizes[0]]
 * row-major), b_0, W_1, b_1, ... (pas_mlp_n_params floats). The object keeps
 * float32 master weights and bf16 working copies: batched passes (forward,
 * gradients, training) run as bf16 tensor-core GEMMs with float32 accumulation;
 * single-vector inference (apply, the loop) reads the bf16 weights with float32
 * activations. */

/* n_layers in [1, 8] weight layers; sizes: host int32 [n_layers + 1] widths
 * (sizes[0] = slopes, sizes[n_layers] = modes); max_batch >= 1 bounds the batch
 * of forward / gradients / train. Parameters start at zero, mean 0, inv_std 1. */
pas_status pas_mlp_create(pas_ctx_t ctx, int32_t n_layers, const int32_t* sizes, int32_t max_batch,
                          pas_mlp_t* out);
void pas_mlp_destroy(pas_mlp_t mlp);
/* Number of parameters (packed), -1 for a NULL handle. Host only. */
int64_t pas_mlp_n_params(pas_mlp_t mlp);
/* h_params: host float32 [n_params] packed. set resets the Adam state.
 * Both synchronise. */
pas_status pas_mlp_set_params(pas_mlp_t mlp, const float* h_params);
pas_status pas_mlp_get_params(pas_mlp_t mlp, float* h_params);
/* Input standardisation, host float32 [sizes[0]] each; synchronous. */
pas_status pas_mlp_set_norm(pas_mlp_t mlp, const float* h_mean, const float* h_inv_std);
/* Single vector: d_slopes device float32 [sizes[0]] -> d_out [sizes[L]]. */
pas_status pas_mlp_apply(pas_mlp_t mlp, const float* d_slopes, float* d_out);
/* Batch (tensor cores): d_S device float32 [batch][sizes[0]] raw slopes ->
 * d_out [batch][sizes[L]]. */
pas_status pas_mlp_forward(pas_mlp_t mlp, int32_t batch, const float* d_S, float* d_out);
/* Loss gradient of the batch (d_S as above, d_Y [batch][sizes[L]] targets):
 * d_grad device float32 [n_params] packed; h_loss (may be NULL) receives the
 * loss, which makes the call synchronous. Parameters are not changed. */
pas_status pas_mlp_gradients(pas_mlp_t mlp, int32_t batch, const float* d_S, const float* d_Y,
                             float* d_grad, float* h_loss);
/* n_steps Adam steps over a device-resident data set d_S [n_data][sizes[0]],
 * d_Y [n_data][sizes[L]]: step t uses the samples d_idx[t*batch .. t*batch +
 * batch - 1] (int32 in [0, n_data)) and learning rate d_lr[t], and writes its
 * loss (before the update) to d_loss[t]. All device arrays are caller-owned
 * and must stay valid; the step is captured once as a CUDA graph per (arrays,
 * batch) and replayed. Out-of-range indices read sample 0 and are reported by
 * pas_mlp_check. */
pas_status pas_mlp_train(pas_mlp_t mlp, const float* d_S, const float* d_Y, int32_t n_data,
                         int32_t batch, const int32_t* d_idx, const float* d_lr, int32_t n_steps,
                         float* d_loss);
/* Synchronise, then report and clear the device flags: PAS_ETIMEOUT if a
 * tensor-core pipeline wait gave up, PAS_EINVAL for an out-of-range sample
 * index; *h_fault (may be NULL) = 1 if the loop's last layer produced a
 * non-finite coefficient since the last check (that coefficient's update was
 * replaced by 0). */
pas_status pas_mlp_check(pas_mlp_t mlp, uint32_t* h_fault);
/* One training pair from a residual OPD: opd = amp * d_opd (device float32
 * [Np][Np]); d_slopes [2 n_valid] = pyramid slopes of opd (reference slopes
 * subtracted, no noise); d_coeffs [n_modes] = (1/n_pix) M^T opd, the modal
 * projection for a basis with M^T M = n_pix I. d_work: device float32 scratch
 * of Np*Np + (2 n_sub)^2 elements. */
pas_status pas_mlp_pair(pas_pyr_t pyr, pas_dm_t dm, const float* d_opd, float amp, float* d_work,
                        float* d_slopes, float* d_coeffs);
/* Use `mlp` (NULL: the linear reconstructor again) as the loop's reconstructor
 * from the next step on; sizes must be [2 n_valid, ..., n_modes]. The loop's
 * graph is captured again at the next step. */
pas_status pas_loop_set_mlp(pas_loop_t loop, pas_mlp_t mlp);

/* ---------------------------------------------------------------- calibration
 * One-off set-up on the GPU (Sec. Example: the reconstruction matrix is calibrated
 * before the run; Table 1 modalrec). These calls allocate their own temporaries and
 * return after their work has completed (they synchronise the stream). */

/* Push-pull interaction matrix through one sensor (exactly one of pyr, sh non-NULL;
 * its noise setting is ignored, its slope reference applies to both pushes and
 * cancels): column m = (s(+amp M_m) - s(-amp M_m)) / (2 amp), M_m the DM's mode m
 * at amp nm RMS. d_IM: device FP64 [n_modes][n_slopes] (column m of the
 * n_slopes x n_modes matrix is contiguous), caller-owned. Runs on the DM's stream. */
pas_status pas_calib_interaction_matrix(pas_pyr_t pyr, pas_sh_t sh, pas_dm_t dm, double amp_nm, double* d_IM);

/* FP64 pseudo-inverse by one-sided Jacobi SVD (Hestenes): A is m x n column-major
 * (d_A[j*m + i] = A(i, j)), m >= n; d_P receives A^+ as n x m row-major
 * (d_P[i*m + k]), singular values below rcond * sigma_max dropped. Optional host
 * outputs: h_sv[n] the singular values (descending), h_rank the number kept,
 * h_sweeps the Jacobi sweeps run. PAS_ETIMEOUT if the rotations do not settle in
 * 60 sweeps. Runs on the context's stream. */
pas_status pas_pinv_f64(pas_ctx_t ctx, const double* d_A, int32_t m, int32_t n, double rcond, double* d_P,
                        double* h_sv, int32_t* h_rank, int32_t* h_sweeps);

/* FP64 product for the set-up (Gram matrices, basis changes):
 * C[i*ldc + k] = sum_j X[i*sxi + j*sxj] * w[j] * Y[k*syk + j*syj] (w NULL: 1), i < ni,
 * k < nk, j < nj; element strides in elements, all device FP64. Asynchronous on the
 * context's stream. */
pas_status pas_gemm_f64(pas_ctx_t ctx, const double* d_X, int64_t sxi, int64_t sxj, const double* d_Y,
                        int64_t syk, int64_t syj, const double* d_w, int32_t ni, int32_t nk, int32_t nj,
                        double* d_C, int64_t ldc);

/* FP32 throughput probe (no counterpart in the paper): the denominator of the FP32
 * roofline quoted for the FFT passes. Launches n_blocks CTAs of 256 threads, each
 * thread running 8 independent FMA chains for `iters` rounds and writing one float
 * to d_sink (device float32 [n_blocks * 256], caller-owned); *h_flops receives the
 * floating-point operations the launch performs (2 per FMA). Asynchronous on
 * cuda_stream (NULL: the legacy default stream); the caller times it with events. */
pas_status pas_fp32_fma_probe(void* cuda_stream, float* d_sink, int32_t n_blocks, int32_t iters,
                              int64_t* h_flops);

/* BF16 tensor-core GEMM (the kernel behind the batched network passes):
 * C[M][N] = A[M][K] * B[N][K]^T, A and B device bf16 (raw uint16 bits)
 * row-major with leading dimensions lda, ldb (multiples of 8, base 16-byte
 * aligned), C device float32 with leading dimension ldc; float32 accumulation.
 * tile_n: output tile width 16, 32, 64, 128 or 256, 0 = automatic. d_err: device
 * uint32 that receives a nonzero code if a pipeline wait timed out. */
pas_status pas_gemm_bf16(pas_ctx_t ctx, int32_t M, int32_t N, int32_t K, const uint16_t* d_A,
                         int32_t lda, const uint16_t* d_B, int32_t ldb, float* d_C, int32_t ldc,
                         int32_t tile_n, uint32_t* d_err);
/* pas_gemm_bf16 whose pipeline waits (a TMA slot to fill or drain, the products to
 * complete) each give up after wait_limit tries of mbarrier.try_wait (0: at once).
 * A wait that gives up sets bits in *d_err (1 producer, 2 product issue,
 * 4 epilogue; 8 if the unwinding itself timed out) and the CTA unwinds: it waits,
 * with the long default bound, for its own copies in flight and the products it
 * issued, frees its tensor memory and returns; C is then unspecified. The failure
 * path of the bounded waits, exercised by the tests; pas_gemm_bf16 uses the default
 * bound (2^22 tries, seconds). */
pas_status pas_gemm_bf16_waits(pas_ctx_t ctx, int32_t M, int32_t N, int32_t K, const uint16_t* d_A,
                               int32_t lda, const uint16_t* d_B, int32_t ldb, float* d_C, int32_t ldc,
                               int32_t tile_n, uint32_t wait_limit, uint32_t* d_err);

#ifdef __cplusplus
}
#endif
#endif /* PAS_H */
