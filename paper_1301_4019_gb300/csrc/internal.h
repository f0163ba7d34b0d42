// internal.h -- launchers shared between the translation units of the library (host side).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rsk {

// Grid-barrier state of a handle's cooperative kernels: the arrival counter (0 between
// launches) and the longest a barrier waits before it gives up with RS_ERR_TIMEOUT.
struct GridBar {
  unsigned int count;
  unsigned int pad;
  unsigned long long timeout_ns;
};
constexpr unsigned long long kDefaultBarrierTimeoutNs = 10ull * 1000 * 1000 * 1000;  // 10 s

// Device-side state of the scan-based schemes (one per handle).
struct ScanGlob {
  double M;                  // max log-weight of the current call
  double S_d;                // total of the max-shifted weights (binary64 view)
  unsigned int ticket_max;   // last-CTA counters (self-resetting)
  unsigned int ticket_tile;
  unsigned int ticket_iscan;
  unsigned int batch_next;   // work counter of the batched kernel (self-resetting)
  unsigned int batch_ticket;
  GridBar bar;               // grid barrier of the cooperative kernels
  int all_zero;              // every weight of the call is zero (set with the total)
  float guide_step;          // W^N / N and N / W^N in binary32 (multinomial guide table),
  float guide_inv_step;      //   set with the total so that no later kernel divides
  unsigned int pad[3];
  double2 S_raw;             // total, in the accumulator type of the call
  double2 scale_raw;         // N / total, in the accumulator type of the call
};

// Optional per-kernel timing: while enabled, an event is recorded on the call's stream
// before every kernel launch and after the last kernel of every call, with a label.
struct Trace {
  cudaEvent_t* ev;
  const char** lbl;
  int n;
  int pos;
};
inline void trace_mark(Trace* t, const char* label, cudaStream_t st) {
  if (t && t->pos < t->n) {
    cudaEventRecord(t->ev[t->pos], st);
    t->lbl[t->pos] = label;
    ++t->pos;
  }
}

constexpr int64_t kBatchMaxN = 1 << 20;  // particles of one filter of a batched call, at most

// Launch shape of a particle-parallel batched kernel: threads per CTA and particles per thread
// (rs_set_batched_launch / rs_tune_batched). The results never depend on it.
struct LaunchCfg {
  int block;
  int ipt;
};
constexpr int kCfgMetropolisF32 = 0, kCfgMetropolisF64 = 1, kCfgPermute = 2, kCfgCount = 3;
constexpr int kMaxTunedBlock = 512;
constexpr int kMaxTunedIpt = 16;

struct Scratch {
  Trace* trace;      // nullptr unless tracing is enabled
  int32_t* d;        // claim vector (Prepermute), max_n
  int32_t* a_tmp;    // unpermuted ancestors, max_n
  void* W;           // cumulative weights of the multinomial scheme, 8 * max_n bytes
  int32_t* guide;    // guide table of the multinomial search, max_n + 1
  double2* rec;      // per-segment records, then prefixes (two blocks of seg_cap(max_tiles))
  double* blockmax;  // per-CTA maxima of the max pass
  long long* irec;   // per-tile records of the integer scan (2 * (max_tiles + 2))
  ScanGlob* glob;
  int* err;          // device status word
  // batched resampling: per-filter and per-tile records
  int32_t* batch_tile_start;  // max_filters + 1
  long long* batch_fmax;      // max_filters
  double2* batch_fS;          // max_filters
  double2* batch_fscale;      // max_filters
  double* batch_fSd;          // max_filters
  double2* batch_s_rec;       // kWarps * batch_tile_cap (one per segment)
  double2* batch_P_rec;       // kWarps * batch_tile_cap + max_filters
  int64_t max_filters;        // max(1024, max_n / 16)
  int64_t batch_tile_cap;     // max_n / kTile + max_filters + 1
  int64_t max_n;
  int64_t max_tiles;
  int max_blocks;    // grid of the max pass
  int coop;          // the device supports cooperative launches
  int launch_mode;   // RS_LAUNCH_AUTO / RS_LAUNCH_FUSED / RS_LAUNCH_SEPARATE
  LaunchCfg batch_cfg[kCfgCount];  // batched Metropolis (binary32, binary64) and Permute
};

// Accumulation of the scan-based schemes: binary32, two-float over binary32 inputs,
// double-float over binary64 inputs (binary32 pipes), native binary64 (FP64 pipe).
enum class Acc { F32, F32C, F64, F64N };

struct Keys;

// scan.cu (fused: the three passes as one cooperative kernel, see fused.cu)
cudaError_t launch_scan_resample(const Scratch& s, int scheme, Acc acc, const void* logw,
                                 int64_t N, uint64_t seed, uint64_t step, uint32_t filter,
                                 int32_t* a_out, int32_t* d_or_null, bool fused,
                                 cudaStream_t st, uint8_t* cl_or_null = nullptr);
cudaError_t launch_cumulative_weights(const Scratch& s, Acc acc, const void* logw, int64_t N,
                                      void* W_out, double* log_total, cudaStream_t st);
cudaError_t launch_cumulative_weights_f64(const Scratch& s, Acc acc, const void* logw, int64_t N,
                                          double* W_out, double* log_total, cudaStream_t st);

// fused.cu: max, tile sums, tile prefixes and emission in one cooperative launch;
// fused_available is false when the device cannot launch it.
bool fused_available(const Scratch& s, int scheme, Acc acc);
cudaError_t launch_fused_passes(const Scratch& s, int scheme, Acc acc, const void* logw,
                                int64_t N, const Keys& keys, int32_t* a_out, int32_t* d,
                                uint8_t* cl, cudaStream_t st);

// batched.cu
cudaError_t launch_batched(const Scratch& s, int scheme, Acc acc, const void* logw,
                           const int64_t* offsets, int F, const int32_t* Bf, int32_t B,
                           uint64_t seed, uint64_t step, double log_wmax, int64_t max_trials,
                           const uint8_t* resample_flags, int32_t* out, int permute,
                           cudaStream_t st);

// mcmc.cu (d, when given, is set to the sentinel N by the launch itself)
cudaError_t launch_metropolis(const Scratch& s, bool f64, const void* logw, int64_t N,
                              int32_t B, uint64_t seed, uint64_t step, uint32_t filter,
                              int32_t* a_out, int32_t* d_or_null, cudaStream_t st);
// (lwmax_dev: the bound read on the device instead of log_wmax, an estimated bound of -inf
// giving the identity, flagged RS_ERR_ZERO_WEIGHT)
cudaError_t launch_rejection(const Scratch& s, bool f64, const void* logw, int64_t N,
                             double log_wmax, bool clamp, int64_t max_trials, uint64_t seed,
                             uint64_t step, uint32_t filter, int32_t* a_out,
                             int32_t* d_or_null, cudaStream_t st,
                             const double* lwmax_dev = nullptr);
// The estimated rejection bound (largest of `sample` drawn log-weights) to *est; *viol = 0.
cudaError_t launch_estimate_bound(const Scratch& s, bool f64, const void* logw, int64_t N,
                                  int64_t sample, uint64_t seed, uint64_t step, uint32_t filter,
                                  double* est, unsigned long long* viol, cudaStream_t st);
// aux.cu: a cooperative launch whose grid barrier expects one arrival more than the grid
// makes, so that every CTA's bounded wait runs out (RS_ERR_TIMEOUT) and the kernel ends.
cudaError_t launch_barrier_timeout_probe(const Scratch& s, cudaStream_t st);
// Self-checks of the acceptance tests (mode 0: binary32 band, every delta; mode 1: binary64
// decisions on n log-weight pairs): the number of wrong decisions goes to *count.
cudaError_t launch_check_acceptance(int mode, int64_t n, unsigned long long* count,
                                    cudaStream_t st);
// scan.cu: self-check of the plain binary32 scans' exponential over every binary32 t <= 0
// (count of results outside the bound; the largest relative error for t >= -87).
cudaError_t launch_check_weight_exp(double bound, unsigned long long* count, double* max_rel,
                                    cudaStream_t st);
// (lvmax_dev: the bound read on the device; viol: count of log-weights above it)
cudaError_t launch_prc_weights(const Scratch& s, bool f64, const void* logw, const int32_t* c,
                               int64_t N, double log_vmax, void* out, cudaStream_t st,
                               const double* lvmax_dev = nullptr,
                               unsigned long long* viol = nullptr);

// noalloc.cu: the static scratch's address for the current device, looked up once
int noalloc_prepare_current_device();

// aux.cu
cudaError_t launch_fill(int32_t* p, int64_t N, int32_t v, cudaStream_t st);
cudaError_t launch_prepermute(const Scratch& s, const int32_t* a, int64_t N, int32_t* d,
                              bool init, cudaStream_t st);
cudaError_t launch_permute(const Scratch& s, const int32_t* a, const int32_t* d, int64_t N,
                           int32_t* c, cudaStream_t st);
// Permute of a non-decreasing ancestry (stratified, systematic) from the claimed bits cl of
// its emission instead of the claims d
cudaError_t launch_permute_sorted_bits(const Scratch& s, const int32_t* a, const uint8_t* cl,
                                       int64_t N, int32_t* c, cudaStream_t st);
cudaError_t launch_offspring(const Scratch& s, const int32_t* a, int64_t N, int32_t* o,
                             cudaStream_t st);
cudaError_t launch_inclusive_scan_i32(const Scratch& s, const int32_t* o, int64_t N,
                                      int32_t* O, cudaStream_t st);
cudaError_t launch_adjacent_difference(const int32_t* O, int64_t N, int32_t* o,
                                       cudaStream_t st);
cudaError_t launch_cumoff_to_ancestors(const Scratch& s, const int32_t* O, int64_t N,
                                       int32_t* a, cudaStream_t st);

// ess.cu (cooperative; cudaErrorNotSupported without cooperative launches)
cudaError_t launch_ess(const Scratch& s, bool f64, const void* logw, int64_t N, double* ess,
                       double* log_total, cudaStream_t st);

// model.cu
cudaError_t launch_copy_ancestors_batched(const Scratch& s, float* x, int D, const int32_t* c,
                                          const int64_t* offsets, int F, cudaStream_t st);
cudaError_t launch_lgssm_step_batched(const Scratch& s, float* x, const int64_t* offsets, int F,
                                      int init, int accumulate, float phi, float sigma_x,
                                      const float* y, float sigma_y, uint64_t seed,
                                      uint64_t step, float* logw, cudaStream_t st);
cudaError_t launch_set_if_below(cudaGraphConditionalHandle hnd, const double* v, double thr,
                                cudaStream_t st);
cudaError_t launch_noop(cudaStream_t st);
cudaError_t launch_mark_resampled(const Scratch& s, float* logw, int64_t N, double* base,
                                  double log_n, int32_t* count, cudaStream_t st);
cudaError_t launch_loglik_step(const Scratch& s, const double* lse, double* base, double* ll,
                               int32_t* count, double c, double log_n, int first,
                               cudaStream_t st);
// Per-filter statistics of a batch's weights (one CTA per filter); null outputs are skipped.
struct WeightStatsOut {
  double* log_total;  // max logw + log sum w
  double* ess;        // (sum w)^2 / sum w^2
  double* beta;       // mean w / max w
  int32_t* B;         // Eq. B for beta and log_eps
  double log_eps;
  uint8_t* below;     // 1 where ess < below_frac * n (0 for empty or all-zero filters)
  double below_frac;
};
cudaError_t launch_reset_logw_batched(const Scratch& s, float* logw, const int64_t* offsets,
                                      int F, const uint8_t* flags, cudaStream_t st);
cudaError_t launch_weight_stats_batched(const Scratch& s, bool f64, const void* logw,
                                        const int64_t* offsets, int F, const WeightStatsOut& o,
                                        cudaStream_t st);
cudaError_t launch_copy_ancestors(const Scratch& s, float* x, int D, const int32_t* c, int64_t N,
                                  cudaStream_t st);
cudaError_t launch_lgssm_step(const Scratch& s, float* x, int64_t N, int init, int accumulate,
                              float phi, float sigma_x, float y, float sigma_y, uint64_t seed,
                              uint64_t step, uint32_t filter, float* logw, cudaStream_t st);

}  // namespace rsk
