// Loop control (Sec. Structure: the loop control object triggers every processing
// object once per simulation step; Table 2: loop.add in run order, loop.run).
// One step on the device, in the order atmo -> prop (residual with the DM layer)
// -> pyr -> ccd -> slopec -> modalrec -> control; the DM layer of step t carries the
// command of step t - delay. The step is captured once as a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <vector>

#include "atmo_dm.cuh"
#include "batchrec.cuh"
#include "internal.h"
#include "mlp.cuh"
#include "psf.cuh"
#include "pyr.cuh"
#include "recon.cuh"
#include "sh.cuh"

struct pas_loop_s {
  pas_ctx_t ctx = nullptr;
  pas_atmo_t atmo = nullptr;
  pas_pyr_t pyr = nullptr;
  pas_sh_t sh = nullptr;    // a Shack-Hartmann loop: the sensor in place of the pyramid
  pas_recon_t rec = nullptr;
  pas_dm_t dm = nullptr;
  pas_mlp_t mlp = nullptr;  // learned reconstructor in place of rec (optional)
  int delay = 1, hist = 1, n_m = 0, n_slopes = 0, nd = 0, Np = 0, n_tiles = 0;
  int batches = 0;          // live batches whose captured graph holds this loop's step
  int n_int = 1;            // detector steps per frame (pas_loop_set_integration)
  int taps = PAS_TAPS_AUTO;         // the atmosphere's tap staging and wait bound at creation
  uint32_t tap_wait_limit = 0;
  // a PSF camera inside the step (pas_loop_attach_camera): its two passes run on a
  // stream of their own after the residual, beside the sensor, and join before the
  // reconstruction (which advances the step counter they read)
  pas_psf_t cam = nullptr;
  float* d_cam_psf = nullptr;
  double* d_cam_sr = nullptr;
  int cam_sr_len = 1;
  long long cam_start = 0;
  cudaStream_t cam_stream = nullptr;
  cudaEvent_t cam_fork = nullptr, cam_join = nullptr;
  float* d_acc = nullptr;   // [nd*nd] the integrating detector's accumulator
  float* d_opd = nullptr;
  float* d_frame = nullptr;
  float* d_slopes = nullptr;
  float* d_dmodes = nullptr;
  float* d_ring = nullptr;
  float* d_cmd = nullptr;
  float* d_gain = nullptr;
  double* d_wfe = nullptr;
  double2* d_wfe_part = nullptr;
  long long* d_step = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // profiling graph: the same step with event-record nodes between the kernels
  cudaGraph_t prof_graph = nullptr;
  cudaGraphExec_t prof_exec = nullptr;
  cudaEvent_t prof_ev[PAS_LOOP_KERNELS + 1] = {};
};

// The step's first kernel: residual = atmosphere - M c (the residual kernel samples
// the wind-shifted layers at its pupil pixels while its other warps stream the basis).
static pas_status enqueue_residual(pas_loop_t L, cudaStream_t st) {
  pas::ResArgs ra = pas::make_res_args(L->dm);
  pas::res_args_set_atmo(ra, L->atmo, L->taps, L->tap_wait_limit);
  ra.opd_atm = nullptr;
  ra.cmd_ring = L->d_ring;
  ra.delay = L->delay;
  ra.d_step = L->d_step;
  ra.dm_sign = 1.0f;
  ra.out = L->d_opd;
  ra.wfe_part = L->d_wfe_part;
  return pas::residual_launch(L->ctx, ra, st, false);
}

// What the loop adds to its sensor's measurement: the step counter as the noise
// frame counter, the residual-WFE finalisation, the integrating detector.
static pas::LoopExtra loop_extra(pas_loop_t L) {
  pas::LoopExtra fa;
  fa.frame_ctr = L->d_step;
  fa.wfe_part = L->d_wfe_part;
  fa.n_wfe_part = L->n_tiles;
  fa.inv_npix = 1.0 / (double)L->dm->n_pix;
  fa.wfe_hist = L->d_wfe;
  fa.wfe_hist_len = L->hist;
  fa.step = L->d_step;
  fa.acc = L->d_acc;
  fa.n_int = L->n_int;
  return fa;
}

// The step's last kernel: reconstruction and integrator (the network in place of
// the matrix when the loop has one); it advances the step counter.
static pas_status enqueue_recon(pas_loop_t L, cudaStream_t st, bool pdl) {
  pas::ReconArgs rc;
  rc.s = L->d_slopes;
  rc.dmodes = L->d_dmodes;
  rc.gain = L->d_gain;
  rc.ring = L->d_ring;
  rc.delay = L->delay;
  rc.step = L->d_step;
  rc.cmd_last = L->d_cmd;
  rc.step_inc = L->d_step;
  rc.n_int = L->n_int;
  return L->mlp ? pas::mlp_loop_launch(L->mlp, rc, st, pdl) : pas::recon_launch(L->rec, rc, st, pdl);
}

// ev (optional): PAS_LOOP_KERNELS + 1 events recorded before each kernel and
// after the last one. skip_recon: stop after the slopes (a batch reconstructs the
// loops that share a reconstructor together). skip_residual: the residual is
// already in the OPD buffer (a batch's shared-DM residual, ordered before by an
// event); the sensor then starts without programmatic dependence.
static pas_status loop_enqueue(pas_loop_t L, cudaStream_t st, cudaEvent_t* ev = nullptr, bool skip_recon = false,
                               bool skip_residual = false) {
  // inside the step the kernels follow each other programmatically (prologues and
  // constant-matrix prefetches overlap the predecessor), except when events are
  // recorded between them for profiling
  const bool pdl = ev == nullptr;
  if (ev) cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal);
  pas_status s = skip_residual ? PAS_OK : enqueue_residual(L, st);
  if (s != PAS_OK) return s;
  if (L->cam) {  // the camera images this step's residual beside the sensor
    cudaError_t e = cudaEventRecord(L->cam_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(L->cam_stream, L->cam_fork, 0);
    if (e != cudaSuccess) return pas::set_error(L->ctx, PAS_ECUDA, "loop camera fork: %s", cudaGetErrorString(e));
    s = pas::psf_launch(L->cam, L->d_opd, L->d_cam_psf, 1, L->d_cam_sr, L->d_step, L->cam_start, L->cam_sr_len,
                        L->cam_stream);
    if (s != PAS_OK) return s;
    e = cudaEventRecord(L->cam_join, L->cam_stream);
    if (e != cudaSuccess) return pas::set_error(L->ctx, PAS_ECUDA, "loop camera join: %s", cudaGetErrorString(e));
  }
  const pas::LoopExtra fa = loop_extra(L);
  const bool pdl_sensor = pdl && !skip_residual;
  if (L->sh)
    s = pas::sh_launch(L->sh, L->d_opd, L->d_frame, L->d_slopes, st, &fa, pdl_sensor);
  else
    s = pas::pyr_launch(L->pyr, L->d_opd, L->d_frame, L->d_slopes, st, &fa, false, ev ? ev + 1 : nullptr,
                        pdl_sensor);
  if (s != PAS_OK) return s;
  if (L->cam) {
    const cudaError_t e = cudaStreamWaitEvent(st, L->cam_join, 0);
    if (e != cudaSuccess) return pas::set_error(L->ctx, PAS_ECUDA, "loop camera join: %s", cudaGetErrorString(e));
  }
  if (skip_recon) return PAS_OK;
  if (ev) cudaEventRecordWithFlags(ev[4], st, cudaEventRecordExternal);
  s = enqueue_recon(L, st, pdl && !L->cam);
  if (ev) cudaEventRecordWithFlags(ev[5], st, cudaEventRecordExternal);
  return s;
}

extern "C" {

void pas_loop_destroy(pas_loop_t L) {
  if (!L) return;
  if (L->exec) cudaGraphExecDestroy(L->exec);
  if (L->graph) cudaGraphDestroy(L->graph);
  if (L->prof_exec) cudaGraphExecDestroy(L->prof_exec);
  if (L->prof_graph) cudaGraphDestroy(L->prof_graph);
  for (int i = 0; i <= PAS_LOOP_KERNELS; ++i)
    if (L->prof_ev[i]) cudaEventDestroy(L->prof_ev[i]);
  if (L->cam_fork) cudaEventDestroy(L->cam_fork);
  if (L->cam_join) cudaEventDestroy(L->cam_join);
  if (L->cam_stream) cudaStreamDestroy(L->cam_stream);
  pas::dev_free(L->d_opd);
  pas::dev_free(L->d_frame);
  pas::dev_free(L->d_slopes);
  pas::dev_free(L->d_dmodes);
  pas::dev_free(L->d_ring);
  pas::dev_free(L->d_cmd);
  pas::dev_free(L->d_gain);
  pas::dev_free(L->d_wfe);
  pas::dev_free(L->d_wfe_part);
  pas::dev_free(L->d_step);
  pas::dev_free(L->d_acc);
  delete L;
}

// One sensor, pyramid or Shack-Hartmann, is given.
static pas_status loop_create(pas_ctx_t ctx, pas_atmo_t atmo, pas_pyr_t pyr, pas_sh_t sh, pas_recon_t rec,
                              pas_dm_t dm, const float* d_gain, int32_t delay, int32_t wfe_history,
                              pas_loop_t* out) {
  if (!ctx || !atmo || !(pyr || sh) || !rec || !dm || !d_gain || !out)
    return pas::set_global_error(PAS_EINVAL, "pas_loop_create: NULL argument");
  *out = nullptr;
  PAS_CHECK_ARG(ctx, delay >= 1 && delay <= 64 && wfe_history >= 1, "pas_loop_create: bad delay or history");
  PAS_CHECK_ARG(ctx, atmo->args.Np == dm->Np, "pas_loop_create: atmosphere and DM pupil sizes differ");
  PAS_CHECK_ARG(ctx, rec->n_modes == dm->n_modes, "pas_loop_create: reconstructor and DM mode counts differ");
  const int n_slopes = sh ? pas::sh_n_slopes(sh) : 2 * pas_pyr_n_valid(pyr);
  PAS_CHECK_ARG(ctx, rec->n_slopes == n_slopes, "pas_loop_create: reconstructor slopes != 2 n_valid");
  PAS_CHECK_ARG(ctx, !sh || pas::sh_np(sh) == dm->Np, "pas_loop_create: sensor and DM pupil sizes differ");
  pas_loop_t L = new pas_loop_s();
  L->ctx = ctx;
  L->atmo = atmo;
  L->taps = atmo->taps;
  L->tap_wait_limit = atmo->wait_limit;
  L->pyr = pyr;
  L->sh = sh;
  L->rec = rec;
  L->dm = dm;
  L->delay = delay;
  L->hist = wfe_history;
  L->n_m = dm->n_modes;
  L->n_slopes = rec->n_slopes;
  L->nd = sh ? pas::sh_frame_side(sh) : pas::pyr_nd(pyr);  // side of the detector frame
  L->Np = dm->Np;
  L->n_tiles = pas::residual_tiles(dm->n_pix);
  pas_status st = PAS_OK;
  auto A = [&](void** p, size_t bytes) {
    if (st == PAS_OK) st = pas::dev_alloc(ctx, p, bytes);
  };
  A((void**)&L->d_opd, sizeof(float) * L->Np * L->Np);
  A((void**)&L->d_frame, sizeof(float) * L->nd * L->nd);
  A((void**)&L->d_slopes, sizeof(float) * L->n_slopes);
  A((void**)&L->d_dmodes, sizeof(float) * L->n_m);
  A((void**)&L->d_ring, sizeof(float) * L->n_m * delay);
  A((void**)&L->d_cmd, sizeof(float) * L->n_m);
  A((void**)&L->d_gain, sizeof(float) * L->n_m);
  A((void**)&L->d_wfe, sizeof(double) * wfe_history);
  A((void**)&L->d_wfe_part, sizeof(double2) * L->n_tiles);
  A((void**)&L->d_step, sizeof(long long));
  if (st != PAS_OK) {
    pas_loop_destroy(L);
    return st;
  }
  cudaError_t e = cudaMemset(L->d_opd, 0, sizeof(float) * L->Np * L->Np);
  if (e == cudaSuccess) e = cudaMemset(L->d_ring, 0, sizeof(float) * L->n_m * delay);
  if (e == cudaSuccess) e = cudaMemset(L->d_cmd, 0, sizeof(float) * L->n_m);
  if (e == cudaSuccess) e = cudaMemset(L->d_wfe, 0, sizeof(double) * wfe_history);
  if (e == cudaSuccess) e = cudaMemset(L->d_step, 0, sizeof(long long));
  if (e == cudaSuccess) e = cudaMemcpy(L->d_gain, d_gain, sizeof(float) * L->n_m, cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) {
    pas_loop_destroy(L);
    return pas::set_error(ctx, PAS_ECUDA, "pas_loop_create: %s", cudaGetErrorString(e));
  }
  *out = L;
  return PAS_OK;
}

pas_status pas_loop_create(pas_ctx_t ctx, pas_atmo_t atmo, pas_pyr_t pyr, pas_recon_t rec, pas_dm_t dm,
                           const float* d_gain, int32_t delay, int32_t wfe_history, pas_loop_t* out) {
  if (!pyr) return pas::set_global_error(PAS_EINVAL, "pas_loop_create: NULL pyramid");
  return loop_create(ctx, atmo, pyr, nullptr, rec, dm, d_gain, delay, wfe_history, out);
}

pas_status pas_loop_create_sh(pas_ctx_t ctx, pas_atmo_t atmo, pas_sh_t sh, pas_recon_t rec, pas_dm_t dm,
                              const float* d_gain, int32_t delay, int32_t wfe_history, pas_loop_t* out) {
  if (!sh) return pas::set_global_error(PAS_EINVAL, "pas_loop_create_sh: NULL sensor");
  return loop_create(ctx, atmo, nullptr, sh, rec, dm, d_gain, delay, wfe_history, out);
}

static pas_status loop_capture(pas_loop_t L) {
  pas_ctx_t ctx = L->ctx;
  // the capture stream must see everything queued before on the context stream
  PAS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  PAS_CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
  pas_status s = loop_enqueue(L, ctx->capture_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &g);
  if (s != PAS_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return pas::set_error(ctx, PAS_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&L->exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return pas::set_error(ctx, PAS_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  L->graph = g;
  return PAS_OK;
}

static pas_status loop_stats(pas_loop_t L, pas_loop_stats* h) {
  pas_ctx_t ctx = L->ctx;
  long long step = 0;
  PAS_CUDA_TRY(ctx, cudaMemcpyAsync(&step, L->d_step, sizeof(step), cudaMemcpyDeviceToHost, ctx->stream));
  PAS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  h->step = step;
  h->wfe_nm = 0.0;
  if (step > 0) {
    PAS_CUDA_TRY(ctx, cudaMemcpy(&h->wfe_nm, L->d_wfe + (step - 1) % L->hist, sizeof(double),
                                 cudaMemcpyDeviceToHost));
  }
  return PAS_OK;
}

pas_status pas_loop_step(pas_loop_t L, int32_t n_steps, pas_loop_stats* h_stats) {
  if (!L) return pas::set_global_error(PAS_EINVAL, "pas_loop_step: NULL loop");
  PAS_CHECK_ARG(L->ctx, n_steps >= 0, "pas_loop_step: negative step count");
  if (!L->exec && n_steps > 0) {
    pas_status s = loop_capture(L);
    if (s != PAS_OK) return s;
  }
  for (int t = 0; t < n_steps; ++t) PAS_CUDA_TRY(L->ctx, cudaGraphLaunch(L->exec, L->ctx->stream));
  if (h_stats) return loop_stats(L, h_stats);
  return PAS_OK;
}

pas_status pas_loop_step_eager(pas_loop_t L, int32_t n_steps) {
  if (!L) return pas::set_global_error(PAS_EINVAL, "pas_loop_step_eager: NULL loop");
  PAS_CHECK_ARG(L->ctx, n_steps >= 0, "pas_loop_step_eager: negative step count");
  for (int t = 0; t < n_steps; ++t) {
    pas_status s = loop_enqueue(L, L->ctx->stream);
    if (s != PAS_OK) return s;
  }
  return PAS_OK;
}

pas_status pas_loop_profile(pas_loop_t L, int32_t n_steps, float* h_ms, int32_t cap, int32_t* n_kernels) {
  if (!L || !h_ms) return pas::set_global_error(PAS_EINVAL, "pas_loop_profile: NULL argument");
  PAS_CHECK_ARG(L->ctx, n_steps >= 1 && cap >= PAS_LOOP_KERNELS, "pas_loop_profile: bad n_steps or cap");
  if (L->sh) return pas::set_error(L->ctx, PAS_ESTATE, "pas_loop_profile: the kernel list is the pyramid loop's");
  pas_ctx_t ctx = L->ctx;
  if (!L->prof_exec) {
    for (int i = 0; i <= PAS_LOOP_KERNELS; ++i) PAS_CUDA_TRY(ctx, cudaEventCreate(&L->prof_ev[i]));
    PAS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    PAS_CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
    pas_status s = loop_enqueue(L, ctx->capture_stream, L->prof_ev);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &g);
    if (s != PAS_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return pas::set_error(ctx, PAS_ECUDA, "profile capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&L->prof_exec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return pas::set_error(ctx, PAS_ECUDA, "profile instantiate: %s", cudaGetErrorString(e));
    }
    L->prof_graph = g;
  }
  double acc[PAS_LOOP_KERNELS] = {0};
  for (int t = 0; t < n_steps; ++t) {
    PAS_CUDA_TRY(ctx, cudaGraphLaunch(L->prof_exec, ctx->stream));
    PAS_CUDA_TRY(ctx, cudaEventSynchronize(L->prof_ev[PAS_LOOP_KERNELS]));
    for (int k = 0; k < PAS_LOOP_KERNELS; ++k) {
      float ms = 0.f;
      PAS_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, L->prof_ev[k], L->prof_ev[k + 1]));
      acc[k] += ms;
    }
  }
  for (int k = 0; k < PAS_LOOP_KERNELS; ++k) h_ms[k] = (float)(acc[k] / n_steps);
  if (n_kernels) *n_kernels = PAS_LOOP_KERNELS;
  return PAS_OK;
}

// Drop the captured graphs (the next step captures the new configuration).
static void loop_drop_graphs(pas_loop_t L) {
  if (L->exec) cudaGraphExecDestroy(L->exec);
  if (L->graph) cudaGraphDestroy(L->graph);
  if (L->prof_exec) cudaGraphExecDestroy(L->prof_exec);
  if (L->prof_graph) cudaGraphDestroy(L->prof_graph);
  L->exec = nullptr;
  L->graph = nullptr;
  L->prof_exec = nullptr;
  L->prof_graph = nullptr;
}

// A batch captured its loops' steps at creation: re-configuring a member would leave
// the batch's graph stepping the old configuration (or reading a detached camera's
// buffers).
#define PAS_LOOP_NOT_BATCHED(L, what)                                                                 \
  do {                                                                                              \
    if ((L)->batches > 0)                                                                           \
      return pas::set_error((L)->ctx, PAS_ESTATE, what ": the loop belongs to a batch (destroy it first)"); \
  } while (0)

pas_status pas_loop_set_integration(pas_loop_t L, int32_t n_int) {
  if (!L) return pas::set_global_error(PAS_EINVAL, "pas_loop_set_integration: NULL loop");
  PAS_LOOP_NOT_BATCHED(L, "pas_loop_set_integration");
  PAS_CHECK_ARG(L->ctx, n_int >= 1 && n_int <= (1 << 20), "pas_loop_set_integration: 1 <= n_int <= 2^20");
  if (n_int > 1 && L->mlp)
    return pas::set_error(L->ctx, PAS_ESTATE, "pas_loop_set_integration: a loop with the linear reconstructor only");
  PAS_CUDA_TRY(L->ctx, cudaStreamSynchronize(L->ctx->stream));
  if (n_int > 1 && !L->d_acc) {
    pas_status st = pas::dev_alloc(L->ctx, (void**)&L->d_acc, sizeof(float) * L->nd * L->nd);
    if (st != PAS_OK) return st;
  }
  if (L->d_acc) PAS_CUDA_TRY(L->ctx, cudaMemset(L->d_acc, 0, sizeof(float) * L->nd * L->nd));
  loop_drop_graphs(L);
  L->n_int = n_int;
  return PAS_OK;
}

pas_status pas_loop_attach_camera(pas_loop_t L, pas_psf_t psf, float* d_psf, double* d_sr, int32_t sr_len,
                                  int64_t start_step) {
  if (!L) return pas::set_global_error(PAS_EINVAL, "pas_loop_attach_camera: NULL loop");
  PAS_LOOP_NOT_BATCHED(L, "pas_loop_attach_camera");
  if (psf) {
    PAS_CHECK_ARG(L->ctx, d_psf != nullptr && sr_len >= 1 && start_step >= 0,
                  "pas_loop_attach_camera: a PSF buffer, sr_len >= 1, start_step >= 0");
    PAS_CHECK_ARG(L->ctx, pas::psf_np(psf) == L->Np, "pas_loop_attach_camera: camera and loop pupil sizes differ");
  }
  PAS_CUDA_TRY(L->ctx, cudaStreamSynchronize(L->ctx->stream));
  if (psf && !L->cam_stream) {
    PAS_CUDA_TRY(L->ctx, cudaStreamCreateWithFlags(&L->cam_stream, cudaStreamNonBlocking));
    PAS_CUDA_TRY(L->ctx, cudaEventCreateWithFlags(&L->cam_fork, cudaEventDisableTiming));
    PAS_CUDA_TRY(L->ctx, cudaEventCreateWithFlags(&L->cam_join, cudaEventDisableTiming));
  }
  loop_drop_graphs(L);
  L->cam = psf;
  L->d_cam_psf = psf ? d_psf : nullptr;
  L->d_cam_sr = psf ? d_sr : nullptr;
  L->cam_sr_len = psf ? sr_len : 1;
  L->cam_start = psf ? start_step : 0;
  return PAS_OK;
}

pas_status pas_loop_set_mlp(pas_loop_t L, pas_mlp_t m) {
  if (!L) return pas::set_global_error(PAS_EINVAL, "pas_loop_set_mlp: NULL loop");
  PAS_LOOP_NOT_BATCHED(L, "pas_loop_set_mlp");
  if (m)
    PAS_CHECK_ARG(L->ctx, m->sz[0] == L->n_slopes && m->sz[m->L] == L->n_m,
                  "pas_loop_set_mlp: network sizes must be [2 n_valid, ..., n_modes]");
  if (m && L->n_int > 1)
    return pas::set_error(L->ctx, PAS_ESTATE, "pas_loop_set_mlp: the loop's detector integrates several steps");
  PAS_CUDA_TRY(L->ctx, cudaStreamSynchronize(L->ctx->stream));
  loop_drop_graphs(L);
  L->mlp = m;
  return PAS_OK;
}

const char* pas_loop_kernel_name(int32_t idx) {
  static const char* names[PAS_LOOP_KERNELS] = {"residual_kernel", "pyr_rows_kernel", "pyr_cols_kernel",
                                                "slopes_kernel", "recon_kernel"};
  return (idx >= 0 && idx < PAS_LOOP_KERNELS) ? names[idx] : nullptr;
}

pas_status pas_loop_buffers(pas_loop_t L, float** opd_res, float** frame, float** slopes, float** dmodes,
                            float** cmd, double** wfe) {
  if (!L) return pas::set_global_error(PAS_EINVAL, "pas_loop_buffers: NULL loop");
  if (opd_res) *opd_res = L->d_opd;
  if (frame) *frame = L->d_frame;
  if (slopes) *slopes = L->d_slopes;
  if (dmodes) *dmodes = L->d_dmodes;
  if (cmd) *cmd = L->d_cmd;
  if (wfe) *wfe = L->d_wfe;
  return PAS_OK;
}

pas_status pas_loop_get_state(pas_loop_t L, int64_t* step, float* h_cmd_ring) {
  if (!L || !step) return pas::set_global_error(PAS_EINVAL, "pas_loop_get_state: NULL argument");
  long long s = 0;
  PAS_CUDA_TRY(L->ctx, cudaStreamSynchronize(L->ctx->stream));
  PAS_CUDA_TRY(L->ctx, cudaMemcpy(&s, L->d_step, sizeof(s), cudaMemcpyDeviceToHost));
  *step = s;
  if (h_cmd_ring)
    PAS_CUDA_TRY(L->ctx, cudaMemcpy(h_cmd_ring, L->d_ring, sizeof(float) * L->n_m * L->delay,
                                    cudaMemcpyDeviceToHost));
  return PAS_OK;
}

pas_status pas_loop_set_state(pas_loop_t L, int64_t step, const float* h_cmd_ring) {
  if (!L || !h_cmd_ring) return pas::set_global_error(PAS_EINVAL, "pas_loop_set_state: NULL argument");
  PAS_CHECK_ARG(L->ctx, step >= 0, "pas_loop_set_state: negative step");
  long long s = step;
  PAS_CUDA_TRY(L->ctx, cudaStreamSynchronize(L->ctx->stream));
  PAS_CUDA_TRY(L->ctx, cudaMemcpy(L->d_step, &s, sizeof(s), cudaMemcpyHostToDevice));
  PAS_CUDA_TRY(L->ctx, cudaMemcpy(L->d_ring, h_cmd_ring, sizeof(float) * L->n_m * L->delay,
                                  cudaMemcpyHostToDevice));
  // the last command is the ring slot of step - 1
  const int slot = (int)(((step - 1) % L->delay + L->delay) % L->delay);
  PAS_CUDA_TRY(L->ctx, cudaMemcpy(L->d_cmd, L->d_ring + (size_t)slot * L->n_m, sizeof(float) * L->n_m,
                                  cudaMemcpyDeviceToDevice));
  // an integrating detector starts an empty frame
  if (L->d_acc) PAS_CUDA_TRY(L->ctx, cudaMemset(L->d_acc, 0, sizeof(float) * L->nd * L->nd));
  return PAS_OK;
}

// ---------------------------------------------------------------- batches

struct pas_batch_s {
  pas_ctx_t ctx = nullptr;
  std::vector<pas_loop_t> loops;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // loops sharing one bfloat16 reconstructor: one tensor-core product per group
  std::vector<std::vector<int>> groups;
  std::vector<pas::BatchRecGroup*> rec_groups;
  std::vector<cudaStream_t> group_streams;
  std::vector<cudaEvent_t> group_join;
  int kernels_per_step = 0;
  // persistent mode: the pyramid loops' rows and columns passes in one launch per
  // transform length (member[i]: loop i's index in it, -1 for a loop stepped whole)
  pas::PyrBatch* pyr_batch = nullptr;
  std::vector<int> member;
  std::vector<cudaEvent_t> res_join;
  std::vector<cudaStream_t> pstreams;  // one per persistent launch
  std::vector<cudaEvent_t> pdone;
  // loops sharing a DM object: one batched residual per group (one basis pass)
  std::vector<std::vector<int>> rgroups;
  std::vector<int> rgroup_of;
  std::vector<pas::ResBatch*> res_batches;
  std::vector<cudaStream_t> rstreams;
  std::vector<cudaEvent_t> rdone;
  bool registered = false;  // the loops count this batch (pas_loop_s::batches)
};

void pas_batch_destroy(pas_batch_t b) {
  if (!b) return;
  if (b->registered)
    for (pas_loop_t L : b->loops) --L->batches;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : b->group_streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->group_join)
    if (e) cudaEventDestroy(e);
  for (pas::BatchRecGroup* g : b->rec_groups) pas::batch_rec_destroy(g);
  for (cudaEvent_t e : b->res_join)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : b->pstreams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->pdone)
    if (e) cudaEventDestroy(e);
  pas::pyr_batch_destroy(b->pyr_batch);
  for (pas::ResBatch* r : b->res_batches) pas::res_batch_destroy(r);
  for (cudaStream_t s : b->rstreams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->rdone)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

pas_status pas_batch_create_ex(pas_ctx_t ctx, pas_loop_t* loops, int32_t n_loops, uint32_t flags,
                               pas_batch_t* out) {
  if (!ctx || !loops || !out) return pas::set_global_error(PAS_EINVAL, "pas_batch_create: NULL argument");
  *out = nullptr;
  PAS_CHECK_ARG(ctx, n_loops >= 1 && n_loops <= 4096, "pas_batch_create: 1 <= n_loops <= 4096");
  PAS_CHECK_ARG(ctx, (flags & ~(uint32_t)PAS_BATCH_PERSISTENT) == 0, "pas_batch_create: unknown flag");
  for (int i = 0; i < n_loops; ++i) {
    PAS_CHECK_ARG(ctx, loops[i] != nullptr, "pas_batch_create: NULL loop");
    for (int j = 0; j < i; ++j) {
      PAS_CHECK_ARG(ctx, loops[j] != loops[i], "pas_batch_create: a loop appears twice");
      // a sensor keeps one measurement's intermediates: loops stepped side by side
      // need one each
      PAS_CHECK_ARG(ctx, (loops[i]->pyr == nullptr || loops[j]->pyr != loops[i]->pyr) &&
                             (loops[i]->sh == nullptr || loops[j]->sh != loops[i]->sh),
                    "pas_batch_create: two loops share a sensor object");
    }
  }
  pas_batch_t b = new pas_batch_s();
  b->ctx = ctx;
  b->loops.assign(loops, loops + n_loops);
  b->streams.assign(n_loops, nullptr);
  b->join.assign(n_loops, nullptr);
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < n_loops && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    pas_batch_destroy(b);
    return pas::set_error(ctx, PAS_ECUDA, "pas_batch_create: %s", cudaGetErrorString(e));
  }
  // loops that share a bfloat16 reconstructor (one frame per step, no network) are
  // reconstructed together: group them by reconstructor, in loop order
  std::vector<int> group_of(n_loops, -1);
  for (int i = 0; i < n_loops; ++i) {
    pas_loop_t L = b->loops[i];
    if (group_of[i] >= 0 || L->mlp || L->n_int != 1 || L->rec->prec != PAS_BF16) continue;
    std::vector<int> members{i};
    for (int j = i + 1; j < n_loops; ++j) {
      pas_loop_t M = b->loops[j];
      if (M->rec == L->rec && !M->mlp && M->n_int == 1) members.push_back(j);
    }
    if (members.size() < 2) continue;
    for (size_t q = 0; q < members.size(); q += 128) {  // at most 128 loops per product
      std::vector<int> part(members.begin() + q, members.begin() + std::min(members.size(), q + 128));
      if (part.size() < 2) continue;
      for (int k : part) group_of[k] = (int)b->groups.size();
      b->groups.push_back(part);
    }
  }
  const size_t n_rec_groups = b->groups.size();
  // loops that share one network: one batched forward per step. A network keeps one
  // set of intermediates, so its loops must all fit one group.
  for (int i = 0; i < n_loops; ++i) {
    pas_loop_t L = b->loops[i];
    if (group_of[i] >= 0 || !L->mlp) continue;
    std::vector<int> members{i};
    for (int j = i + 1; j < n_loops; ++j)
      if (b->loops[j]->mlp == L->mlp) members.push_back(j);
    if (members.size() < 2) continue;
    if ((int)members.size() > std::min(128, L->mlp->max_batch)) {
      pas_batch_destroy(b);
      return pas::set_error(ctx, PAS_EINVAL,
                            "pas_batch_create: %zu loops share a network of batch size %d (at most min(128, it))",
                            members.size(), L->mlp->max_batch);
    }
    for (int k : members) group_of[k] = (int)b->groups.size();
    b->groups.push_back(members);
  }
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    const std::vector<int>& grp = b->groups[gi];
    std::vector<const float*> sl;
    std::vector<float*> ring, cmd, dm;
    std::vector<const float*> gain;
    std::vector<long long*> step;
    std::vector<int> delay;
    for (int k : grp) {
      pas_loop_t L = b->loops[k];
      sl.push_back(L->d_slopes);
      ring.push_back(L->d_ring);
      gain.push_back(L->d_gain);
      cmd.push_back(L->d_cmd);
      dm.push_back(L->d_dmodes);
      step.push_back(L->d_step);
      delay.push_back(L->delay);
    }
    pas::BatchRecGroup* g = nullptr;
    pas_status sg =
        gi < n_rec_groups
            ? pas::batch_rec_create(ctx, b->loops[grp[0]]->rec, (int)grp.size(), sl.data(), ring.data(), gain.data(),
                                    cmd.data(), dm.data(), step.data(), delay.data(), &g)
            : pas::batch_mlp_create(ctx, b->loops[grp[0]]->mlp, (int)grp.size(), sl.data(), ring.data(), gain.data(),
                                    cmd.data(), dm.data(), step.data(), delay.data(), &g);
    if (sg != PAS_OK) {
      pas_batch_destroy(b);
      return sg;
    }
    b->rec_groups.push_back(g);
    cudaStream_t gs = nullptr;
    cudaEvent_t ge = nullptr;
    e = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ge, cudaEventDisableTiming);
    b->group_streams.push_back(gs);
    b->group_join.push_back(ge);
    if (e != cudaSuccess) {
      pas_batch_destroy(b);
      return pas::set_error(ctx, PAS_ECUDA, "pas_batch_create: %s", cudaGetErrorString(e));
    }
  }
  // loops sharing a DM object whose sources are at infinity: one residual pass over
  // the basis per group, in loop order
  b->rgroup_of.assign(n_loops, -1);
  for (int i = 0; i < n_loops; ++i) {
    pas_loop_t L = b->loops[i];
    if (b->rgroup_of[i] >= 0 || !pas::res_batch_ok(L->atmo->args)) continue;
    std::vector<int> members{i};
    for (int j = i + 1; j < n_loops; ++j)
      if (b->loops[j]->dm == L->dm && pas::res_batch_ok(b->loops[j]->atmo->args)) members.push_back(j);
    if (members.size() < 2) continue;
    std::vector<pas::ResBatchLoop> rl;
    for (int k : members) {
      pas_loop_t M = b->loops[k];
      pas::ResBatchLoop r;
      r.atmo = M->atmo->args;
      r.cmd_ring = M->d_ring;
      r.delay = M->delay;
      r.d_step = M->d_step;
      r.out = M->d_opd;
      r.wfe_part = M->d_wfe_part;
      rl.push_back(r);
    }
    pas::ResBatch* rb = nullptr;
    pas_status sr = pas::res_batch_create(ctx, L->dm, (int)rl.size(), rl.data(), &rb);
    if (sr != PAS_OK) {
      pas_batch_destroy(b);
      return sr;
    }
    for (int k : members) b->rgroup_of[k] = (int)b->rgroups.size();
    b->rgroups.push_back(members);
    b->res_batches.push_back(rb);
    cudaStream_t rs = nullptr;
    cudaEvent_t re = nullptr;
    e = cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&re, cudaEventDisableTiming);
    b->rstreams.push_back(rs);
    b->rdone.push_back(re);
    if (e != cudaSuccess) {
      pas_batch_destroy(b);
      return pas::set_error(ctx, PAS_ECUDA, "pas_batch_create: %s", cudaGetErrorString(e));
    }
  }
  b->member.assign(n_loops, -1);
  if (flags & PAS_BATCH_PERSISTENT) {
    std::vector<pas_pyr_t> py;
    std::vector<const float*> opd;
    std::vector<float*> frame, sl;
    std::vector<pas::LoopExtra> ex;
    for (int i = 0; i < n_loops; ++i) {
      pas_loop_t L = b->loops[i];
      if (!L->pyr) continue;
      if (L->cam) {
        pas_batch_destroy(b);
        return pas::set_error(ctx, PAS_EINVAL, "pas_batch_create: a loop with an attached camera in a persistent batch");
      }
      b->member[i] = (int)py.size();
      py.push_back(L->pyr);
      opd.push_back(L->d_opd);
      frame.push_back(L->d_frame);
      sl.push_back(L->d_slopes);
      ex.push_back(loop_extra(L));
    }
    if (!py.empty()) {
      pas_status sp = pas::pyr_batch_create(ctx, (int)py.size(), py.data(), opd.data(), frame.data(), sl.data(),
                                            ex.data(), &b->pyr_batch);
      if (sp != PAS_OK) {
        pas_batch_destroy(b);
        return sp;
      }
    }
    b->res_join.assign(n_loops, nullptr);
    for (int i = 0; i < n_loops && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->res_join[i], cudaEventDisableTiming);
    const int np = b->pyr_batch ? pas::pyr_batch_n_groups(b->pyr_batch) : 0;
    b->pstreams.assign(np, nullptr);
    b->pdone.assign(np, nullptr);
    for (int g = 0; g < np && e == cudaSuccess; ++g) {
      e = cudaStreamCreateWithFlags(&b->pstreams[g], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->pdone[g], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
      pas_batch_destroy(b);
      return pas::set_error(ctx, PAS_ECUDA, "pas_batch_create: %s", cudaGetErrorString(e));
    }
  }
  b->kernels_per_step = 0;
  for (int i = 0; i < n_loops; ++i) {
    // a persistent member launches its residual and slopes kernels (and its
    // reconstruction unless its group's product does it)
    const int whole = b->member[i] >= 0 ? 3 : b->loops[i]->sh ? 3 : PAS_LOOP_KERNELS;
    const int recon = b->loops[i]->mlp ? b->loops[i]->mlp->L : 1;  // a network: one launch per layer
    b->kernels_per_step += whole - 1 + (group_of[i] >= 0 ? 0 : recon) - (b->rgroup_of[i] >= 0 ? 1 : 0) +
                           (b->loops[i]->cam ? 2 : 0);
  }
  for (pas::BatchRecGroup* g : b->rec_groups) b->kernels_per_step += pas::batch_rec_kernels(g);
  b->kernels_per_step += 2 * (int)b->rgroups.size();
  if (b->pyr_batch) b->kernels_per_step += pas::pyr_batch_n_groups(b->pyr_batch);
  // one graph per step: every loop's step is a branch of its own (fork on the
  // context's capture stream, one stream per loop, join back); a group's product
  // follows the slopes of all its loops on a stream of its own
  for (pas_loop_t L : b->loops) {
    cudaError_t s0 = cudaStreamSynchronize(L->ctx->stream);
    if (s0 != cudaSuccess) {
      pas_batch_destroy(b);
      return pas::set_error(ctx, PAS_ECUDA, "pas_batch_create: %s", cudaGetErrorString(s0));
    }
  }
  cudaStream_t cs = ctx->capture_stream;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  pas_status st = PAS_OK;
  if (e == cudaSuccess) e = cudaEventRecord(b->fork, cs);
  // the shared-DM residuals first, each on a stream of its own
  for (size_t g = 0; g < b->rgroups.size() && e == cudaSuccess && st == PAS_OK; ++g) {
    e = cudaStreamWaitEvent(b->rstreams[g], b->fork, 0);
    if (e == cudaSuccess) st = pas::res_batch_launch(b->res_batches[g], b->rstreams[g]);
    if (e == cudaSuccess && st == PAS_OK) e = cudaEventRecord(b->rdone[g], b->rstreams[g]);
    if (e == cudaSuccess && st == PAS_OK) e = cudaStreamWaitEvent(cs, b->rdone[g], 0);
  }
  for (int i = 0; i < n_loops && e == cudaSuccess && st == PAS_OK; ++i) {
    const int rg = b->rgroup_of[i];
    e = cudaStreamWaitEvent(b->streams[i], rg >= 0 ? b->rdone[rg] : b->fork, 0);
    if (b->member[i] >= 0) {  // its residual; its persistent launch follows
      if (rg >= 0) continue;
      if (e == cudaSuccess) st = enqueue_residual(b->loops[i], b->streams[i]);
      if (e == cudaSuccess && st == PAS_OK) e = cudaEventRecord(b->res_join[i], b->streams[i]);
      continue;
    }
    if (e == cudaSuccess) st = loop_enqueue(b->loops[i], b->streams[i], nullptr, group_of[i] >= 0, rg >= 0);
    if (e == cudaSuccess && st == PAS_OK) e = cudaEventRecord(b->join[i], b->streams[i]);
    if (e == cudaSuccess && st == PAS_OK && group_of[i] < 0) e = cudaStreamWaitEvent(cs, b->join[i], 0);
  }
  if (b->pyr_batch && e == cudaSuccess && st == PAS_OK) {
    // one persistent launch per transform length, on a stream of its own after the
    // residuals of its loops; each loop's slopes and reconstruction after its launch
    for (size_t g = 0; g < b->pstreams.size() && e == cudaSuccess && st == PAS_OK; ++g) {
      for (int i = 0; i < n_loops && e == cudaSuccess; ++i) {
        if (b->member[i] < 0 || pas::pyr_batch_group_of(b->pyr_batch, b->member[i]) != (int)g) continue;
        const int rg = b->rgroup_of[i];
        e = cudaStreamWaitEvent(b->pstreams[g], rg >= 0 ? b->rdone[rg] : b->res_join[i], 0);
      }
      if (e == cudaSuccess) st = pas::pyr_batch_launch_group(b->pyr_batch, (int)g, b->pstreams[g]);
      if (e == cudaSuccess && st == PAS_OK) e = cudaEventRecord(b->pdone[g], b->pstreams[g]);
      if (e == cudaSuccess && st == PAS_OK) e = cudaStreamWaitEvent(cs, b->pdone[g], 0);
    }
    for (int i = 0; i < n_loops && e == cudaSuccess && st == PAS_OK; ++i) {
      if (b->member[i] < 0) continue;
      e = cudaStreamWaitEvent(b->streams[i], b->pdone[pas::pyr_batch_group_of(b->pyr_batch, b->member[i])], 0);
      if (e == cudaSuccess) st = pas::pyr_batch_slopes(b->pyr_batch, b->member[i], b->streams[i], false);
      if (e == cudaSuccess && st == PAS_OK && group_of[i] < 0) st = enqueue_recon(b->loops[i], b->streams[i], true);
      if (e == cudaSuccess && st == PAS_OK) e = cudaEventRecord(b->join[i], b->streams[i]);
      if (e == cudaSuccess && st == PAS_OK && group_of[i] < 0) e = cudaStreamWaitEvent(cs, b->join[i], 0);
    }
  }
  for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess && st == PAS_OK; ++gi) {
    cudaStream_t gs = b->group_streams[gi];
    for (int k : b->groups[gi])
      if (e == cudaSuccess) e = cudaStreamWaitEvent(gs, b->join[k], 0);
    if (e == cudaSuccess) st = pas::batch_rec_launch(b->rec_groups[gi], gs);
    if (e == cudaSuccess && st == PAS_OK) e = cudaEventRecord(b->group_join[gi], gs);
    if (e == cudaSuccess && st == PAS_OK) e = cudaStreamWaitEvent(cs, b->group_join[gi], 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  if (e == cudaSuccess) e = e2;
  if (st == PAS_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
  b->graph = g;
  if (st != PAS_OK || e != cudaSuccess) {
    pas_batch_destroy(b);
    if (st != PAS_OK) return st;
    return pas::set_error(ctx, PAS_ECUDA, "pas_batch_create capture: %s", cudaGetErrorString(e));
  }
  for (pas_loop_t L : b->loops) ++L->batches;
  b->registered = true;
  *out = b;
  return PAS_OK;
}

pas_status pas_batch_create(pas_ctx_t ctx, pas_loop_t* loops, int32_t n_loops, pas_batch_t* out) {
  return pas_batch_create_ex(ctx, loops, n_loops, 0u, out);
}

pas_status pas_batch_step(pas_batch_t b, int32_t n_steps) {
  if (!b) return pas::set_global_error(PAS_EINVAL, "pas_batch_step: NULL batch");
  PAS_CHECK_ARG(b->ctx, n_steps >= 0, "pas_batch_step: negative step count");
  for (int t = 0; t < n_steps; ++t) PAS_CUDA_TRY(b->ctx, cudaGraphLaunch(b->exec, b->ctx->stream));
  return PAS_OK;
}

int32_t pas_batch_size(pas_batch_t b) { return b ? (int32_t)b->loops.size() : -1; }

int32_t pas_batch_kernels_per_step(pas_batch_t b) { return b ? b->kernels_per_step : -1; }

int32_t pas_batch_n_groups(pas_batch_t b) { return b ? (int32_t)b->groups.size() : -1; }

pas_status pas_batch_check(pas_batch_t b, uint32_t* h_fault) {
  if (!b) return pas::set_global_error(PAS_EINVAL, "pas_batch_check: NULL batch");
  unsigned int f = 0;
  for (pas::BatchRecGroup* g : b->rec_groups) {
    unsigned int x = 0;
    PAS_CUDA_TRY(b->ctx, cudaMemcpy(&x, pas::batch_rec_err(g), sizeof(x), cudaMemcpyDeviceToHost));
    f |= x;
    if (x) PAS_CUDA_TRY(b->ctx, cudaMemset(pas::batch_rec_err(g), 0, sizeof(unsigned int)));
  }
  unsigned int w = 0;
  if (b->pyr_batch) {
    unsigned int* d = pas::pyr_batch_err(b->pyr_batch);
    PAS_CUDA_TRY(b->ctx, cudaMemcpy(&w, d, sizeof(w), cudaMemcpyDeviceToHost));
    if (w) PAS_CUDA_TRY(b->ctx, cudaMemset(d, 0, sizeof(unsigned int)));
  }
  if (h_fault) *h_fault = f | (w ? 0x100u : 0u);
  if (f) return pas::set_error(b->ctx, PAS_ETIMEOUT, "batched reconstruction: a product's wait gave up (%u)", f);
  if (w) return pas::set_error(b->ctx, PAS_ETIMEOUT, "persistent pyramid launch: a columns task's wait gave up");
  return PAS_OK;
}

pas_status pas_batch_persistent_geometry(pas_batch_t b, int32_t g, int32_t* h_geo) {
  if (!b || !h_geo) return pas::set_global_error(PAS_EINVAL, "pas_batch_persistent_geometry: NULL argument");
  PAS_CHECK_ARG(b->ctx, b->pyr_batch && g >= 0 && g < pas::pyr_batch_n_groups(b->pyr_batch),
                "pas_batch_persistent_geometry: no such persistent launch");
  pas::pyr_batch_geometry(b->pyr_batch, g, h_geo);
  return PAS_OK;
}

int32_t pas_batch_n_residual_groups(pas_batch_t b) { return b ? (int32_t)b->rgroups.size() : -1; }

int32_t pas_batch_n_persistent(pas_batch_t b) {
  return b ? (b->pyr_batch ? pas::pyr_batch_n_groups(b->pyr_batch) : 0) : -1;
}

pas_status pas_batch_set_wait_limit(pas_batch_t b, int64_t polls) {
  if (!b) return pas::set_global_error(PAS_EINVAL, "pas_batch_set_wait_limit: NULL batch");
  PAS_CHECK_ARG(b->ctx, b->pyr_batch != nullptr, "pas_batch_set_wait_limit: not a persistent batch");
  PAS_CHECK_ARG(b->ctx, polls >= 0, "pas_batch_set_wait_limit: negative limit");
  const long long v = polls;
  PAS_CUDA_TRY(b->ctx, cudaStreamSynchronize(b->ctx->stream));
  PAS_CUDA_TRY(b->ctx, cudaMemcpy(pas::pyr_batch_wait_limit(b->pyr_batch), &v, sizeof(v), cudaMemcpyHostToDevice));
  return PAS_OK;
}

pas_status pas_batch_probe_waits(pas_batch_t b, uint32_t* h_fault) {
  if (!b) return pas::set_global_error(PAS_EINVAL, "pas_batch_probe_waits: NULL batch");
  PAS_CHECK_ARG(b->ctx, b->pyr_batch != nullptr, "pas_batch_probe_waits: not a persistent batch");
  cudaStream_t st = b->ctx->stream;
  PAS_CUDA_TRY(b->ctx, cudaStreamSynchronize(st));
  pas_status s = pas::pyr_batch_launch(b->pyr_batch, st, true);
  if (s != PAS_OK) return s;
  PAS_CUDA_TRY(b->ctx, cudaStreamSynchronize(st));
  return pas_batch_check(b, h_fault);
}

}  // extern "C"
