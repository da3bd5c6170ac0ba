// hse_eval.cu -- C-ABI evaluation entry points: input checks, cell list,
// real-space part, Fourier-space part and their combination (Sec. 4:
// u = u_R + u_F + self term).
#include "hse_internal.cuh"

namespace hse {
hse_status launch_validate_strengths(hse_plan p, int64_t n, const double* str, cudaStream_t s);
}

using namespace hse;

static hse_status prepare_sources(hse_plan p, int64_t n_src, const double* src, const double* str, int64_t n_tgt,
                                  const double* tgt, bool need_str, cudaStream_t s) {
  if (n_src < 0 || n_tgt < 0) return set_err(p, HSE_ERR_INVALID, "negative count");
  if (n_src > 0x1fffffff) return set_err(p, HSE_ERR_UNSUPPORTED, "n_src above 2^29 - 1");
  if (n_src > 0 && (!src || (need_str && !str))) return set_err(p, HSE_ERR_INVALID, "NULL source array");
  if (!tgt && n_tgt != n_src) return set_err(p, HSE_ERR_INVALID, "targets = sources needs n_tgt == n_src");
  if (tgt == nullptr && n_tgt > 0 && !src) return set_err(p, HSE_ERR_INVALID, "NULL source array");
  HSE_TRY(ensure_workspace(p, n_src));
  HSE_CUDA(p, cudaMemsetAsync(p->ws.flag, 0, sizeof(int), s));
  HSE_TRY(launch_validate(p, n_src, src, 1, s));
  if (need_str) HSE_TRY(launch_validate_strengths(p, n_src, str, s));
  if (tgt) HSE_TRY(launch_validate(p, n_tgt, tgt, 0, s));
  HSE_TRY(read_flag(p, s, "input check"));
  stage_mark(p, HSE_STAGE_CELLS, s);
  if (n_src == 0) return HSE_OK;
  HSE_TRY(build_cell_list(p, n_src, src, nullptr, nullptr, nullptr, s));
  return gather_sorted(p, n_src, src, need_str ? str : nullptr, s);
}

static hse_status ensure_overlap_streams(hse_plan p) {
  if (p->s_real) return HSE_OK;
  int lo = 0, hi = 0;
  HSE_CUDA(p, cudaDeviceGetStreamPriorityRange(&lo, &hi));
  HSE_CUDA(p, cudaStreamCreateWithPriority(&p->s_real, cudaStreamNonBlocking, lo));
  HSE_CUDA(p, cudaStreamCreateWithPriority(&p->s_four, cudaStreamNonBlocking, hi));
  HSE_CUDA(p, cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
  HSE_CUDA(p, cudaEventCreateWithFlags(&p->ev_real, cudaEventDisableTiming));
  HSE_CUDA(p, cudaEventCreateWithFlags(&p->ev_four, cudaEventDisableTiming));
  return HSE_OK;
}

static hse_status eval_impl(hse_plan p, int64_t n_src, const double* src, const double* str, int64_t n_tgt,
                            const double* tgt, double* u_real, double* u_four, void* stream) {
  if (!p) return HSE_ERR_INVALID;
  p->err.clear();
  if (!p->grid_ready && u_four) return set_err(p, HSE_ERR_INVALID, "grid size M not set (hse_plan_set_grid)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n_tgt > 0 && !u_real && !u_four) return set_err(p, HSE_ERR_INVALID, "no output array");
  p->n_launch = 0;
  p->n_fft = 0;
  p->ev_recorded = false;
  stage_mark(p, HSE_STAGE_CHECK, s);
  HSE_TRY(prepare_sources(p, n_src, src, str, n_tgt, tgt, true, s));
  if (n_tgt == 0) return HSE_OK;
  if (n_src == 0) {
    if (u_real) HSE_CUDA(p, cudaMemsetAsync(u_real, 0, sizeof(double) * 3 * n_tgt, s));
    if (u_four) HSE_CUDA(p, cudaMemsetAsync(u_four, 0, sizeof(double) * 3 * n_tgt, s));
    return HSE_OK;
  }
  p->last_overlap = false;
  if (p->overlap && u_real && u_four) {
    // The two halves share only read-only inputs: run them concurrently, the
    // Fourier part at higher priority, and let its gather (which adds into
    // out when out is shared) wait for the real part.
    HSE_TRY(ensure_overlap_streams(p));
    HSE_CUDA(p, cudaEventRecord(p->ev_fork, s));
    HSE_CUDA(p, cudaStreamWaitEvent(p->s_real, p->ev_fork, 0));
    HSE_CUDA(p, cudaStreamWaitEvent(p->s_four, p->ev_fork, 0));
    stage_mark(p, HSE_STAGE_REAL, p->s_real);
    HSE_TRY(real_space(p, n_src, n_tgt, tgt, u_real, false, p->s_real));
    if (p->timing) HSE_CUDA(p, cudaEventRecord(p->ev_real_end, p->s_real));
    HSE_CUDA(p, cudaEventRecord(p->ev_real, p->s_real));
    stage_mark(p, HSE_STAGE_SPREAD, p->s_four);
    HSE_TRY(fourier_space(p, n_src, n_tgt, tgt, u_four, u_four == u_real, p->s_four,
                          u_four == u_real ? p->ev_real : nullptr));
    stage_mark(p, HSE_N_STAGES, p->s_four);
    HSE_CUDA(p, cudaEventRecord(p->ev_four, p->s_four));
    HSE_CUDA(p, cudaStreamWaitEvent(s, p->ev_real, 0));
    HSE_CUDA(p, cudaStreamWaitEvent(s, p->ev_four, 0));
    p->last_overlap = true;
    p->ev_recorded = p->timing;
    return HSE_OK;
  }
  stage_mark(p, HSE_STAGE_REAL, s);
  if (u_real) HSE_TRY(real_space(p, n_src, n_tgt, tgt, u_real, false, s));
  stage_mark(p, HSE_STAGE_SPREAD, s);
  if (u_four) {
    HSE_TRY(fourier_space(p, n_src, n_tgt, tgt, u_four, u_four == u_real, s));
  } else {
    for (int i = HSE_STAGE_FFT; i <= HSE_STAGE_GATHER; ++i) stage_mark(p, i, s);
  }
  stage_mark(p, HSE_N_STAGES, s);
  p->ev_recorded = p->timing;
  return HSE_OK;
}

extern "C" hse_status hse_eval(hse_plan p, int64_t n_src, const double* src_xyz, const double* strengths,
                               int64_t n_tgt, const double* tgt_xyz, double* vel, void* cuda_stream) {
  return eval_impl(p, n_src, src_xyz, strengths, n_tgt, tgt_xyz, vel, vel, cuda_stream);
}

extern "C" hse_status hse_eval_parts(hse_plan p, int64_t n_src, const double* src_xyz, const double* strengths,
                                     int64_t n_tgt, const double* tgt_xyz, double* u_real, double* u_fourier,
                                     void* cuda_stream) {
  if (u_real && u_real == u_fourier) return set_err(p, HSE_ERR_INVALID, "u_real and u_fourier alias");
  return eval_impl(p, n_src, src_xyz, strengths, n_tgt, tgt_xyz, u_real, u_fourier, cuda_stream);
}

extern "C" hse_status hse_cell_list(hse_plan p, int64_t n, const double* pos, int32_t* cell_id, int32_t* perm,
                                    int32_t* cell_start, void* cuda_stream) {
  if (!p) return HSE_ERR_INVALID;
  p->err.clear();
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (n < 0 || (n > 0 && (!pos || !cell_id || !perm)) || !cell_start)
    return set_err(p, HSE_ERR_INVALID, "bad arguments");
  if (n > 0x1fffffff) return set_err(p, HSE_ERR_UNSUPPORTED, "n above 2^29 - 1");
  HSE_TRY(ensure_workspace(p, n));
  HSE_CUDA(p, cudaMemsetAsync(p->ws.flag, 0, sizeof(int), s));
  HSE_TRY(launch_validate(p, n, pos, 1, s));
  HSE_TRY(read_flag(p, s, "input check"));
  return build_cell_list(p, n, pos, cell_id, perm, cell_start, s);
}

extern "C" hse_status hse_neighbor_counts(hse_plan p, int64_t n_src, const double* src_xyz, int64_t n_tgt,
                                          const double* tgt_xyz, int32_t* n_pairs, int32_t* n_images,
                                          void* cuda_stream) {
  if (!p) return HSE_ERR_INVALID;
  p->err.clear();
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (n_tgt > 0 && (!n_pairs || !n_images)) return set_err(p, HSE_ERR_INVALID, "NULL output");
  HSE_TRY(prepare_sources(p, n_src, src_xyz, nullptr, n_tgt, tgt_xyz, false, s));
  if (n_tgt == 0) return HSE_OK;
  if (n_src == 0) {
    HSE_CUDA(p, cudaMemsetAsync(n_pairs, 0, sizeof(int32_t) * n_tgt, s));
    HSE_CUDA(p, cudaMemsetAsync(n_images, 0, sizeof(int32_t) * n_tgt, s));
    return HSE_OK;
  }
  return neighbor_counts(p, n_src, n_tgt, tgt_xyz, n_pairs, n_images, s);
}

extern "C" hse_status hse_spread_grids(hse_plan p, int64_t n_src, const double* src_xyz, const double* strengths,
                                       double* grids, int* n_comp, void* cuda_stream) {
  if (!p || !n_comp) return HSE_ERR_INVALID;
  p->err.clear();
  if (!p->grid_ready) return set_err(p, HSE_ERR_INVALID, "grid size M not set (hse_plan_set_grid)");
  *n_comp = paper_components(p->prm.kernel_mask).n;
  if (!grids) return HSE_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  HSE_TRY(prepare_sources(p, n_src, src_xyz, strengths, n_src, nullptr, true, s));
  return spread_paper_grids(p, n_src, grids, s);
}

extern "C" hse_status hse_plan_set_overlap(hse_plan p, int enable) {
  if (!p) return HSE_ERR_INVALID;
  p->overlap = enable != 0;
  return HSE_OK;
}

extern "C" hse_status hse_plan_set_real_residency(hse_plan p, int blocks_per_sm) {
  if (!p) return HSE_ERR_INVALID;
  if (blocks_per_sm < 0 || blocks_per_sm > 64) return set_err(p, HSE_ERR_INVALID, "blocks_per_sm %d", blocks_per_sm);
  if (p->n_sm == 0) {
    int dev = 0;
    HSE_CUDA(p, cudaGetDevice(&dev));
    HSE_CUDA(p, cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev));
  }
  p->real_bps = blocks_per_sm;
  return HSE_OK;
}

extern "C" hse_status hse_plan_set_timing(hse_plan p, int enable) {
  if (!p) return HSE_ERR_INVALID;
  if (enable && !p->timing) {
    for (int i = 0; i <= HSE_N_STAGES; ++i) HSE_CUDA(p, cudaEventCreate(&p->ev[i]));
    HSE_CUDA(p, cudaEventCreate(&p->ev_real_end));
    p->timing = true;
  } else if (!enable && p->timing) {
    cudaDeviceSynchronize();
    for (int i = 0; i <= HSE_N_STAGES; ++i) cudaEventDestroy(p->ev[i]);
    cudaEventDestroy(p->ev_real_end);
    p->timing = false;
  }
  p->ev_recorded = false;
  return HSE_OK;
}

extern "C" hse_status hse_get_eval_stats(hse_plan p, hse_eval_stats* out) {
  if (!p || !out) return HSE_ERR_INVALID;
  out->n_kernel_launches = p->n_launch;
  out->n_fft_execs = p->n_fft;
  out->timing = 0;
  for (int i = 0; i < HSE_N_STAGES; ++i) out->stage_ms[i] = 0.0;
  out->overlapped = p->last_overlap ? 1 : 0;
  out->total_ms = 0.0;
  if (p->timing && p->ev_recorded) {
    HSE_CUDA(p, cudaEventSynchronize(p->ev[HSE_N_STAGES]));
    if (p->last_overlap) HSE_CUDA(p, cudaEventSynchronize(p->ev_real_end));
    for (int i = 0; i < HSE_N_STAGES; ++i) {
      // concurrent halves: the real stage ends at its own event
      cudaEvent_t end = (p->last_overlap && i == HSE_STAGE_REAL) ? p->ev_real_end : p->ev[i + 1];
      float ms = 0.f;
      HSE_CUDA(p, cudaEventElapsedTime(&ms, p->ev[i], end));
      out->stage_ms[i] = ms;
    }
    float tot = 0.f;
    HSE_CUDA(p, cudaEventElapsedTime(&tot, p->ev[HSE_STAGE_CHECK], p->ev[HSE_N_STAGES]));
    out->total_ms = tot;
    out->timing = 1;
  }
  return HSE_OK;
}
