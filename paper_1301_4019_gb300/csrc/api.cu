// api.cu -- the C ABI declared in include/resample.h: handle lifetime, host-side argument
// checks and dispatch to the kernels. No call allocates or synchronises except rs_create,
// rs_destroy and rs_last_error.
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "../../include/resample_measure.h"
#include "common.cuh"
#include "internal.h"
#include "measure.h"

struct rs_handle {
  int device;
  rsk::Scratch s;
  rsk::Trace trace;
  // conditional capture (rs_capture_if_below .. rs_capture_end_if)
  cudaStream_t body_stream;
  cudaStream_t cap_stream;
  bool cap_active;
  int saved_mode;
};

namespace {

constexpr int64_t kMaxN = 2147483647LL;

inline cudaStream_t as_stream(void* p) { return static_cast<cudaStream_t>(p); }

int set_device(const rs_handle* h) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return RS_ERR_CUDA;
  if (cur != h->device && cudaSetDevice(h->device) != cudaSuccess) return RS_ERR_CUDA;
  return RS_OK;
}

int check_n(const rs_handle* h, int64_t N) {
  if (N < 1 || N > kMaxN) return RS_ERR_ARG;
  if (h && N > h->s.max_n) return RS_ERR_CAPACITY;
  return RS_OK;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? RS_OK : RS_ERR_CUDA; }

// Accumulation of the scan-based schemes for a (dtype, precision) pair (checked before).
rsk::Acc accumulation(int dtype, int prec) {
  if (dtype == RS_F64) return prec == RS_PREC_BINARY64 ? rsk::Acc::F64N : rsk::Acc::F64;
  return prec == RS_PREC_COMPENSATED ? rsk::Acc::F32C : rsk::Acc::F32;
}

void end_mark(rs_handle* h, cudaStream_t st) { rsk::trace_mark(h->s.trace, "end", st); }

void clear_trace(rs_handle* h) {
  delete[] h->trace.ev;
  delete[] h->trace.lbl;
  h->trace = rsk::Trace{nullptr, nullptr, 0, 0};
  h->s.trace = nullptr;
}

void free_scratch(rsk::Scratch& s) {
  cudaFree(s.d);
  cudaFree(s.a_tmp);
  cudaFree(s.W);
  cudaFree(s.guide);
  cudaFree(s.rec);
  cudaFree(s.blockmax);
  cudaFree(s.irec);
  cudaFree(s.glob);
  cudaFree(s.err);
  cudaFree(s.batch_tile_start);
  cudaFree(s.batch_fmax);
  cudaFree(s.batch_fS);
  cudaFree(s.batch_fscale);
  cudaFree(s.batch_fSd);
  cudaFree(s.batch_s_rec);
  cudaFree(s.batch_P_rec);
  std::memset(&s, 0, sizeof(s));
}

bool valid_launch(int block, int ipt) {
  return block >= 32 && block <= rsk::kMaxTunedBlock && block % 32 == 0 && ipt >= 1 &&
         ipt <= rsk::kMaxTunedIpt;
}

// Milliseconds of `reps` back-to-back calls of `call` on stream s (CUDA events), after one
// untimed call; a negative value when a call or the timing failed.
template <typename Call>
float time_calls(cudaStream_t s, int reps, Call call) {
  if (call() != RS_OK) return -1.0f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.0f;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.0f;
  }
  float ms = -1.0f;
  bool ok = cudaEventRecord(e0, s) == cudaSuccess;
  for (int r = 0; ok && r < reps; ++r) ok = call() == RS_OK;
  ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
       cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ok ? ms : -1.0f;
}

}  // namespace

extern "C" {

int rs_create(rs_handle** out, int64_t max_n, int device) {
  if (!out || max_n < 1 || max_n > kMaxN) return RS_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return RS_ERR_CUDA;
  rs_handle* h = new (std::nothrow) rs_handle();
  if (!h) return RS_ERR_CUDA;
  h->device = device;
  rsk::Scratch& s = h->s;
  std::memset(&s, 0, sizeof(s));
  s.max_n = max_n;
  s.max_tiles = (max_n + rsk::kTile - 1) / rsk::kTile;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      sms < 1)
    sms = 1;
  s.max_blocks = sms * 8;  // grid of the max pass: 8 CTAs per SM of this device
  s.launch_mode = RS_LAUNCH_AUTO;
  for (int k = 0; k < rsk::kCfgCount; ++k) s.batch_cfg[k] = rsk::LaunchCfg{rsk::kBlock, 1};
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess) coop = 0;
  s.coop = coop;
  // the allocation-free call's static scratch on this device: looked up now, so that calls
  // made later while a stream is captured find it ready
  bool ok = rsk::noalloc_prepare_current_device() == RS_OK;
  ok &= cudaMalloc(&s.d, sizeof(int32_t) * max_n) == cudaSuccess;
  ok &= cudaMalloc(&s.a_tmp, sizeof(int32_t) * max_n) == cudaSuccess;
  ok &= cudaMalloc(&s.W, 8 * static_cast<size_t>(max_n)) == cudaSuccess;
  ok &= cudaMalloc(&s.guide, sizeof(int32_t) * (max_n + 1)) == cudaSuccess;
  ok &= cudaMalloc(&s.rec, sizeof(double2) * 2 * rsk::seg_cap(s.max_tiles)) == cudaSuccess;
  ok &= cudaMalloc(&s.blockmax, sizeof(double) * s.max_blocks) == cudaSuccess;
  ok &= cudaMalloc(&s.irec, sizeof(long long) * 2 * (s.max_tiles + 2)) == cudaSuccess;
  ok &= cudaMalloc(&s.glob, sizeof(rsk::ScanGlob)) == cudaSuccess;
  s.max_filters = max_n / 16 > 1024 ? max_n / 16 : 1024;
  s.batch_tile_cap = max_n / rsk::kTile + s.max_filters + 1;
  const size_t mf = static_cast<size_t>(s.max_filters);
  const size_t tc = static_cast<size_t>(s.batch_tile_cap);
  ok &= cudaMalloc(&s.batch_tile_start, sizeof(int32_t) * (mf + 1)) == cudaSuccess;
  ok &= cudaMalloc(&s.batch_fmax, sizeof(long long) * mf) == cudaSuccess;
  ok &= cudaMalloc(&s.batch_fS, sizeof(double2) * mf) == cudaSuccess;
  ok &= cudaMalloc(&s.batch_fscale, sizeof(double2) * mf) == cudaSuccess;
  ok &= cudaMalloc(&s.batch_fSd, sizeof(double) * mf) == cudaSuccess;
  ok &= cudaMalloc(&s.batch_s_rec, sizeof(double2) * rsk::kWarps * tc) == cudaSuccess;
  ok &= cudaMalloc(&s.batch_P_rec, sizeof(double2) * (rsk::kWarps * tc + mf)) == cudaSuccess;
  ok &= cudaMalloc(&s.err, sizeof(int)) == cudaSuccess;
  if (ok) {
    ok &= cudaMemset(s.glob, 0, sizeof(rsk::ScanGlob)) == cudaSuccess;
    const unsigned long long limit = rsk::kDefaultBarrierTimeoutNs;
    ok &= cudaMemcpy(&s.glob->bar.timeout_ns, &limit, sizeof(limit), cudaMemcpyHostToDevice) ==
          cudaSuccess;
    const int none = rsk::kNoError;
    ok &= cudaMemcpy(s.err, &none, sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaDeviceSynchronize() == cudaSuccess;
  }
  if (ok) ok &= cudaStreamCreateWithFlags(&h->body_stream, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    if (h->body_stream) cudaStreamDestroy(h->body_stream);
    free_scratch(s);
    delete h;
    return RS_ERR_CUDA;
  }
  *out = h;
  return RS_OK;
}

int rs_destroy(rs_handle* h) {
  if (!h) return RS_OK;
  const int st = set_device(h);
  clear_trace(h);
  if (h->body_stream) cudaStreamDestroy(h->body_stream);
  free_scratch(h->s);
  delete h;
  return st;
}

int rs_trace(rs_handle* h, void* const* events, int n) {
  if (!h || n < 0 || (n > 0 && !events)) return RS_ERR_ARG;
  clear_trace(h);
  if (n == 0) return RS_OK;
  h->trace.ev = new (std::nothrow) cudaEvent_t[n];
  h->trace.lbl = new (std::nothrow) const char*[n];
  if (!h->trace.ev || !h->trace.lbl) {
    clear_trace(h);
    return RS_ERR_ARG;
  }
  for (int i = 0; i < n; ++i) {
    h->trace.ev[i] = static_cast<cudaEvent_t>(events[i]);
    h->trace.lbl[i] = nullptr;
  }
  h->trace.n = n;
  h->trace.pos = 0;
  h->s.trace = &h->trace;
  return RS_OK;
}

int rs_trace_count(const rs_handle* h) { return h ? h->trace.pos : 0; }

const char* rs_trace_label(const rs_handle* h, int i) {
  if (!h || i < 0 || i >= h->trace.pos) return nullptr;
  return h->trace.lbl[i];
}

int rs_resample(rs_handle* h, int scheme, int dtype, const void* logw_dev, int64_t N,
                int32_t B, uint64_t seed, uint64_t step, int32_t* ancestors_dev, int permute,
                const rs_opts* opts, void* stream) {
  if (!h || !logw_dev || !ancestors_dev) return RS_ERR_ARG;
  int st = check_n(h, N);
  if (st != RS_OK) return st;
  if (scheme < RS_MULTINOMIAL || scheme > RS_REJECTION) return RS_ERR_ARG;
  if (dtype != RS_F32 && dtype != RS_F64) return RS_ERR_ARG;
  if (permute != 0 && permute != 1) return RS_ERR_ARG;
  rs_opts o;
  o.prec = RS_PREC_PLAIN;
  o.log_wmax = 0.0;
  o.max_trials = 1 << 20;
  o.filter = 0;
  if (opts) o = *opts;
  if (o.prec != RS_PREC_PLAIN && o.prec != RS_PREC_COMPENSATED && o.prec != RS_PREC_BINARY64)
    return RS_ERR_ARG;
  if (o.prec == RS_PREC_BINARY64 && dtype != RS_F64) return RS_ERR_ARG;
  if (!std::isfinite(o.log_wmax)) return RS_ERR_ARG;
  if (o.max_trials < 1 || o.max_trials > 0xFFFFFFFFLL) return RS_ERR_ARG;
  if (o.filter >= (1u << 29)) return RS_ERR_ARG;
  if (scheme == RS_METROPOLIS && B < 0) return RS_ERR_ARG;
  if ((st = set_device(h)) != RS_OK) return st;
  const cudaStream_t s = as_stream(stream);
  const bool f64 = dtype == RS_F64;
  int32_t* a_out = permute ? h->s.a_tmp : ancestors_dev;
  int32_t* d = permute ? h->s.d : nullptr;
  // the stratified / systematic emission gives the sorted Permute its claimed bits (in the
  // claims' buffer) instead of the claims
  uint8_t* cl = nullptr;
  cudaError_t e = cudaSuccess;
  switch (scheme) {
    case RS_MULTINOMIAL:
    case RS_STRATIFIED:
    case RS_SYSTEMATIC: {
      const rsk::Acc acc = accumulation(dtype, o.prec);
      const int mode = h->s.launch_mode;
      const bool fused = mode != RS_LAUNCH_SEPARATE && rsk::fused_available(h->s, scheme, acc);
      if (permute && scheme != RS_MULTINOMIAL) {
        cl = reinterpret_cast<uint8_t*>(h->s.d);
        d = nullptr;
      }
      e = rsk::launch_scan_resample(h->s, scheme, acc, logw_dev, N, seed, step, o.filter, a_out,
                                    d, fused, s, cl);
      break;
    }
    case RS_METROPOLIS:  // (the launch also sets the claims d to the sentinel N)
      e = rsk::launch_metropolis(h->s, f64, logw_dev, N, B, seed, step, o.filter, a_out, d, s);
      break;
    case RS_REJECTION:
      e = rsk::launch_rejection(h->s, f64, logw_dev, N, o.log_wmax, false, o.max_trials, seed,
                                step, o.filter, a_out, d, s);
      break;
  }
  if (e == cudaSuccess && permute) {
    if (cl)  // stratified, systematic: a non-decreasing ancestry
      e = rsk::launch_permute_sorted_bits(h->s, a_out, cl, N, ancestors_dev, s);
    else
      e = rsk::launch_permute(h->s, a_out, d, N, ancestors_dev, s);
  }
  end_mark(h, s);
  return cuda_status(e);
}

int rs_resample_prc(rs_handle* h, int dtype, const void* logw_dev, int64_t N, double log_vmax,
                    int64_t max_trials, uint64_t seed, uint64_t step, uint32_t filter,
                    int32_t* ancestors_dev, void* logw_out_dev, int permute, void* stream) {
  if (!h || !logw_dev || !ancestors_dev || !logw_out_dev) return RS_ERR_ARG;
  int st = check_n(h, N);
  if (st != RS_OK) return st;
  if (dtype != RS_F32 && dtype != RS_F64) return RS_ERR_ARG;
  if (permute != 0 && permute != 1) return RS_ERR_ARG;
  if (!std::isfinite(log_vmax)) return RS_ERR_ARG;
  if (max_trials < 1 || max_trials > 0xFFFFFFFFLL) return RS_ERR_ARG;
  if (filter >= (1u << 29)) return RS_ERR_ARG;
  if (logw_out_dev == logw_dev) return RS_ERR_ARG;
  if ((st = set_device(h)) != RS_OK) return st;
  const cudaStream_t s = as_stream(stream);
  const bool f64 = dtype == RS_F64;
  int32_t* a_out = permute ? h->s.a_tmp : ancestors_dev;
  int32_t* d = permute ? h->s.d : nullptr;
  cudaError_t e = rsk::launch_rejection(h->s, f64, logw_dev, N, log_vmax, true, max_trials,
                                        seed, step, filter, a_out, d, s);
  if (e == cudaSuccess && permute)
    e = rsk::launch_permute(h->s, a_out, d, N, ancestors_dev, s);
  if (e == cudaSuccess)
    e = rsk::launch_prc_weights(h->s, f64, logw_dev, ancestors_dev, N, log_vmax, logw_out_dev,
                                s);
  end_mark(h, s);
  return cuda_status(e);
}

int rs_resample_rejection_estimated(rs_handle* h, int dtype, const void* logw_dev, int64_t N,
                                    int64_t sample, int64_t max_trials, uint64_t seed,
                                    uint64_t step, uint32_t filter, int32_t* ancestors_dev,
                                    void* logw_out_dev, double* log_wmax_dev,
                                    unsigned long long* violations_dev, int permute,
                                    void* stream) {
  if (!h || !logw_dev || !ancestors_dev || !logw_out_dev || !log_wmax_dev || !violations_dev)
    return RS_ERR_ARG;
  int st = check_n(h, N);
  if (st != RS_OK) return st;
  if (dtype != RS_F32 && dtype != RS_F64) return RS_ERR_ARG;
  if (permute != 0 && permute != 1) return RS_ERR_ARG;
  if (sample < 1 || sample > kMaxN) return RS_ERR_ARG;
  if (max_trials < 1 || max_trials > 0xFFFFFFFFLL) return RS_ERR_ARG;
  if (filter >= (1u << 29)) return RS_ERR_ARG;
  if (logw_out_dev == logw_dev) return RS_ERR_ARG;
  if ((st = set_device(h)) != RS_OK) return st;
  const cudaStream_t s = as_stream(stream);
  const bool f64 = dtype == RS_F64;
  int32_t* a_out = permute ? h->s.a_tmp : ancestors_dev;
  int32_t* d = permute ? h->s.d : nullptr;
  cudaError_t e = rsk::launch_estimate_bound(h->s, f64, logw_dev, N, sample, seed, step, filter,
                                             log_wmax_dev, violations_dev, s);
  if (e == cudaSuccess)
    e = rsk::launch_rejection(h->s, f64, logw_dev, N, 0.0, true, max_trials, seed, step, filter,
                              a_out, d, s, log_wmax_dev);
  if (e == cudaSuccess && permute) e = rsk::launch_permute(h->s, a_out, d, N, ancestors_dev, s);
  if (e == cudaSuccess)
    e = rsk::launch_prc_weights(h->s, f64, logw_dev, ancestors_dev, N, 0.0, logw_out_dev, s,
                                log_wmax_dev, violations_dev);
  end_mark(h, s);
  return cuda_status(e);
}

int rs_resample_batched_masked(rs_handle* h, int scheme, int dtype, const void* logw_dev,
                               const int64_t* offsets_dev, int32_t F, const int32_t* B_dev,
                               int32_t B, uint64_t seed, uint64_t step,
                               const uint8_t* resample_dev, int32_t* ancestors_dev, int permute,
                               const rs_opts* opts, void* stream) {
  if (!h || !logw_dev || !offsets_dev || !ancestors_dev) return RS_ERR_ARG;
  if (F < 1) return RS_ERR_ARG;
  if (F > h->s.max_filters) return RS_ERR_CAPACITY;
  if (scheme < RS_MULTINOMIAL || scheme > RS_REJECTION) return RS_ERR_ARG;
  if (dtype != RS_F32 && dtype != RS_F64) return RS_ERR_ARG;
  if (permute != 0 && permute != 1) return RS_ERR_ARG;
  rs_opts o;
  o.prec = RS_PREC_PLAIN;
  o.log_wmax = 0.0;
  o.max_trials = 1 << 20;
  o.filter = 0;
  if (opts) o = *opts;
  if (o.prec != RS_PREC_PLAIN && o.prec != RS_PREC_COMPENSATED && o.prec != RS_PREC_BINARY64)
    return RS_ERR_ARG;
  if (o.prec == RS_PREC_BINARY64 && dtype != RS_F64) return RS_ERR_ARG;
  if (!std::isfinite(o.log_wmax)) return RS_ERR_ARG;
  if (o.max_trials < 1 || o.max_trials > 0xFFFFFFFFLL) return RS_ERR_ARG;
  if (scheme == RS_METROPOLIS && !B_dev && B < 0) return RS_ERR_ARG;
  int st = set_device(h);
  if (st != RS_OK) return st;
  const cudaStream_t s = as_stream(stream);
  const cudaError_t e = rsk::launch_batched(h->s, scheme, accumulation(dtype, o.prec), logw_dev,
                                            offsets_dev, F, B_dev, B, seed, step, o.log_wmax,
                                            o.max_trials, resample_dev, ancestors_dev, permute, s);
  end_mark(h, s);
  return cuda_status(e);
}

int rs_resample_batched(rs_handle* h, int scheme, int dtype, const void* logw_dev,
                        const int64_t* offsets_dev, int32_t F, const int32_t* B_dev, int32_t B,
                        uint64_t seed, uint64_t step, int32_t* ancestors_dev, int permute,
                        const rs_opts* opts, void* stream) {
  return rs_resample_batched_masked(h, scheme, dtype, logw_dev, offsets_dev, F, B_dev, B, seed,
                                    step, nullptr, ancestors_dev, permute, opts, stream);
}

int rs_reset_weights_batched(rs_handle* h, float* logw_dev, const int64_t* offsets_dev,
                             int32_t F, const uint8_t* flags_dev, void* stream) {
  if (!h || !logw_dev || !offsets_dev || !flags_dev || F < 1) return RS_ERR_ARG;
  if (F > INT_MAX / 2) return RS_ERR_ARG;
  int st = set_device(h);
  if (st != RS_OK) return st;
  const cudaError_t e = rsk::launch_reset_logw_batched(h->s, logw_dev, offsets_dev, F, flags_dev,
                                                       as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_cumulative_weights(rs_handle* h, int dtype, int prec, const void* logw_dev, int64_t N,
                          void* W_dev, double* log_total_dev, void* stream) {
  if (!h || !logw_dev || !W_dev) return RS_ERR_ARG;
  int st = check_n(h, N);
  if (st != RS_OK) return st;
  if (dtype != RS_F32 && dtype != RS_F64) return RS_ERR_ARG;
  if (prec != RS_PREC_PLAIN && prec != RS_PREC_COMPENSATED && prec != RS_PREC_BINARY64)
    return RS_ERR_ARG;
  if (prec == RS_PREC_BINARY64 && dtype != RS_F64) return RS_ERR_ARG;
  if ((st = set_device(h)) != RS_OK) return st;
  const rsk::Acc acc = accumulation(dtype, prec);
  const cudaError_t e =
      rsk::launch_cumulative_weights(h->s, acc, logw_dev, N, W_dev, log_total_dev, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_cumulative_weights_f64(rs_handle* h, int dtype, int prec, const void* logw_dev,
                              int64_t N, double* W_dev, double* log_total_dev, void* stream) {
  if (!h || !logw_dev || !W_dev) return RS_ERR_ARG;
  int st = check_n(h, N);
  if (st != RS_OK) return st;
  if (dtype != RS_F32 && dtype != RS_F64) return RS_ERR_ARG;
  if (prec != RS_PREC_PLAIN && prec != RS_PREC_COMPENSATED && prec != RS_PREC_BINARY64)
    return RS_ERR_ARG;
  if (prec == RS_PREC_BINARY64 && dtype != RS_F64) return RS_ERR_ARG;
  if ((st = set_device(h)) != RS_OK) return st;
  const cudaError_t e = rsk::launch_cumulative_weights_f64(
      h->s, accumulation(dtype, prec), logw_dev, N, W_dev, log_total_dev, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_offspring(rs_handle* h, const int32_t* a_dev, int64_t N, int32_t* o_dev, void* stream) {
  if (!h || !a_dev || !o_dev) return RS_ERR_ARG;
  int st = check_n(nullptr, N);
  if (st != RS_OK) return st;
  if ((st = set_device(h)) != RS_OK) return st;
  const cudaError_t e = rsk::launch_offspring(h->s, a_dev, N, o_dev, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_cumulative_offspring(rs_handle* h, const int32_t* o_dev, int64_t N, int32_t* O_dev,
                            void* stream) {
  if (!h || !o_dev || !O_dev) return RS_ERR_ARG;
  int st = check_n(h, N);
  if (st != RS_OK) return st;
  if ((st = set_device(h)) != RS_OK) return st;
  const cudaError_t e = rsk::launch_inclusive_scan_i32(h->s, o_dev, N, O_dev, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_adjacent_difference(rs_handle* h, const int32_t* O_dev, int64_t N, int32_t* o_dev,
                           void* stream) {
  if (!h || !O_dev || !o_dev) return RS_ERR_ARG;
  int st = check_n(nullptr, N);
  if (st != RS_OK) return st;
  if ((st = set_device(h)) != RS_OK) return st;
  rsk::trace_mark(h->s.trace, "adjacent_difference", as_stream(stream));
  const cudaError_t e = rsk::launch_adjacent_difference(O_dev, N, o_dev, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_cumulative_offspring_to_ancestors(rs_handle* h, const int32_t* O_dev, int64_t N,
                                         int32_t* a_dev, void* stream) {
  if (!h || !O_dev || !a_dev) return RS_ERR_ARG;
  int st = check_n(nullptr, N);
  if (st != RS_OK) return st;
  if ((st = set_device(h)) != RS_OK) return st;
  const cudaError_t e = rsk::launch_cumoff_to_ancestors(h->s, O_dev, N, a_dev, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_prepermute(rs_handle* h, const int32_t* a_dev, int64_t N, int32_t* d_dev, void* stream) {
  if (!h || !a_dev || !d_dev) return RS_ERR_ARG;
  int st = check_n(nullptr, N);
  if (st != RS_OK) return st;
  if ((st = set_device(h)) != RS_OK) return st;
  const cudaError_t e = rsk::launch_prepermute(h->s, a_dev, N, d_dev, true, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_permute(rs_handle* h, const int32_t* a_dev, int64_t N, int32_t* c_dev, void* stream) {
  if (!h || !a_dev || !c_dev || a_dev == c_dev) return RS_ERR_ARG;
  int st = check_n(h, N);
  if (st != RS_OK) return st;
  if ((st = set_device(h)) != RS_OK) return st;
  const cudaStream_t s = as_stream(stream);
  cudaError_t e = rsk::launch_prepermute(h->s, a_dev, N, h->s.d, true, s);
  if (e == cudaSuccess) e = rsk::launch_permute(h->s, a_dev, h->s.d, N, c_dev, s);
  end_mark(h, s);
  return cuda_status(e);
}

int rs_set_launch_mode(rs_handle* h, int mode) {
  if (!h || (mode != RS_LAUNCH_AUTO && mode != RS_LAUNCH_FUSED && mode != RS_LAUNCH_SEPARATE))
    return RS_ERR_ARG;
  h->s.launch_mode = mode;
  return RS_OK;
}

int rs_ess(rs_handle* h, int dtype, const void* logw_dev, int64_t N, double* ess_dev,
           double* log_total_dev, void* stream) {
  if (!h || !logw_dev || (!ess_dev && !log_total_dev)) return RS_ERR_ARG;
  int st = check_n(h, N);
  if (st != RS_OK) return st;
  if (dtype != RS_F32 && dtype != RS_F64) return RS_ERR_ARG;
  if ((st = set_device(h)) != RS_OK) return st;
  const cudaError_t e = rsk::launch_ess(h->s, dtype == RS_F64, logw_dev, N, ess_dev,
                                        log_total_dev, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_copy_ancestors(rs_handle* h, float* x_dev, int32_t D, const int32_t* c_dev, int64_t N,
                      void* stream) {
  if (!h || !x_dev || !c_dev || D < 1) return RS_ERR_ARG;
  int st = check_n(nullptr, N);
  if (st != RS_OK) return st;
  if (N > INT64_MAX / D) return RS_ERR_ARG;
  if ((st = set_device(h)) != RS_OK) return st;
  const cudaError_t e = rsk::launch_copy_ancestors(h->s, x_dev, D, c_dev, N, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_lgssm_step(rs_handle* h, float* x_dev, int64_t N, int init, int accumulate, float phi,
                  float sigma_x, float y, float sigma_y, uint64_t seed, uint64_t step,
                  uint32_t filter, float* logw_dev, void* stream) {
  if (!h || !x_dev || !logw_dev) return RS_ERR_ARG;
  int st = check_n(nullptr, N);
  if (st != RS_OK) return st;
  if ((init != 0 && init != 1) || (accumulate != 0 && accumulate != 1)) return RS_ERR_ARG;
  if (!(std::fabs(phi) < 1.0f) || !(sigma_x > 0.0f) || !(sigma_y > 0.0f) || !std::isfinite(y) ||
      !std::isfinite(sigma_x) || !std::isfinite(sigma_y) || filter >= (1u << 29))
    return RS_ERR_ARG;
  if ((st = set_device(h)) != RS_OK) return st;
  const cudaError_t e = rsk::launch_lgssm_step(h->s, x_dev, N, init, accumulate, phi, sigma_x,
                                               y, sigma_y, seed, step, filter, logw_dev,
                                               as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_copy_ancestors_batched(rs_handle* h, float* x_dev, int32_t D, const int32_t* c_dev,
                              const int64_t* offsets_dev, int32_t F, void* stream) {
  if (!h || !x_dev || !c_dev || !offsets_dev || D < 1 || F < 1) return RS_ERR_ARG;
  if (h->s.max_n > INT64_MAX / D) return RS_ERR_ARG;
  int st = set_device(h);
  if (st != RS_OK) return st;
  const cudaError_t e = rsk::launch_copy_ancestors_batched(h->s, x_dev, D, c_dev, offsets_dev,
                                                           F, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_lgssm_step_batched(rs_handle* h, float* x_dev, const int64_t* offsets_dev, int32_t F,
                          int init, int accumulate, float phi, float sigma_x,
                          const float* y_dev, float sigma_y, uint64_t seed, uint64_t step,
                          float* logw_dev, void* stream) {
  if (!h || !x_dev || !offsets_dev || !y_dev || !logw_dev || F < 1) return RS_ERR_ARG;
  if (F > (1 << 29)) return RS_ERR_ARG;  // the filter index must fit counter word 3
  if ((init != 0 && init != 1) || (accumulate != 0 && accumulate != 1)) return RS_ERR_ARG;
  if (!(std::fabs(phi) < 1.0f) || !(sigma_x > 0.0f) || !(sigma_y > 0.0f) ||
      !std::isfinite(sigma_x) || !std::isfinite(sigma_y))
    return RS_ERR_ARG;
  int st = set_device(h);
  if (st != RS_OK) return st;
  const cudaError_t e = rsk::launch_lgssm_step_batched(h->s, x_dev, offsets_dev, F, init,
                                                       accumulate, phi, sigma_x, y_dev, sigma_y,
                                                       seed, step, logw_dev, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_log_sum_weights_batched(rs_handle* h, int dtype, const void* logw_dev,
                               const int64_t* offsets_dev, int32_t F, double* out_dev,
                               void* stream) {
  if (!h || !logw_dev || !offsets_dev || !out_dev || F < 1) return RS_ERR_ARG;
  if (dtype != RS_F32 && dtype != RS_F64) return RS_ERR_ARG;
  if (F > INT_MAX / 2) return RS_ERR_ARG;
  int st = set_device(h);
  if (st != RS_OK) return st;
  rsk::WeightStatsOut o{};
  o.log_total = out_dev;
  const cudaError_t e = rsk::launch_weight_stats_batched(h->s, dtype == RS_F64, logw_dev,
                                                         offsets_dev, F, o, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_ess_batched(rs_handle* h, int dtype, const void* logw_dev, const int64_t* offsets_dev,
                   int32_t F, double* ess_dev, double* log_total_dev, double threshold_frac,
                   uint8_t* below_dev, void* stream) {
  if (!h || !logw_dev || !offsets_dev || (!ess_dev && !log_total_dev && !below_dev) || F < 1)
    return RS_ERR_ARG;
  if (below_dev && !(threshold_frac >= 0.0 && threshold_frac <= 1.0)) return RS_ERR_ARG;
  if (dtype != RS_F32 && dtype != RS_F64) return RS_ERR_ARG;
  if (F > INT_MAX / 2) return RS_ERR_ARG;
  int st = set_device(h);
  if (st != RS_OK) return st;
  rsk::WeightStatsOut o{};
  o.log_total = log_total_dev;
  o.ess = ess_dev;
  o.below = below_dev;
  o.below_frac = threshold_frac;
  const cudaError_t e = rsk::launch_weight_stats_batched(h->s, dtype == RS_F64, logw_dev,
                                                         offsets_dev, F, o, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_metropolis_B_batched(rs_handle* h, int dtype, const void* logw_dev,
                            const int64_t* offsets_dev, int32_t F, double eps, int32_t* B_dev,
                            double* beta_dev, void* stream) {
  if (!h || !logw_dev || !offsets_dev || !B_dev || F < 1) return RS_ERR_ARG;
  if (dtype != RS_F32 && dtype != RS_F64) return RS_ERR_ARG;
  if (!(eps > 0.0 && eps < 1.0)) return RS_ERR_ARG;
  if (F > INT_MAX / 2) return RS_ERR_ARG;
  int st = set_device(h);
  if (st != RS_OK) return st;
  rsk::WeightStatsOut o{};
  o.B = B_dev;
  o.beta = beta_dev;
  o.log_eps = std::log(eps);
  const cudaError_t e = rsk::launch_weight_stats_batched(h->s, dtype == RS_F64, logw_dev,
                                                         offsets_dev, F, o, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}


int rs_philox_throughput(rs_handle* h, int64_t threads, uint32_t draws_per_thread,
                         uint64_t seed, uint32_t* xor_dev, void* stream) {
  if (!h || !xor_dev || threads < 1 || threads > (int64_t{1} << 32) || draws_per_thread < 1)
    return RS_ERR_ARG;
  int st = set_device(h);
  if (st != RS_OK) return st;
  const cudaStream_t s = as_stream(stream);
  rsk::trace_mark(h->s.trace, "philox_throughput", s);
  const cudaError_t e = rsk::launch_philox_throughput(threads, draws_per_thread, seed, xor_dev, s);
  end_mark(h, s);
  return cuda_status(e);
}

int rs_set_barrier_timeout(rs_handle* h, uint64_t timeout_ns) {
  if (!h || timeout_ns == 0) return RS_ERR_ARG;
  int st = set_device(h);
  if (st != RS_OK) return st;
  const unsigned long long v = timeout_ns;
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(&h->s.glob->bar.timeout_ns, &v, sizeof(v), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return RS_ERR_CUDA;
  return RS_OK;
}

int rs_check_barrier_timeout(rs_handle* h, void* stream) {
  if (!h) return RS_ERR_ARG;
  int st = set_device(h);
  if (st != RS_OK) return st;
  if (!h->s.coop) return RS_ERR_CUDA;
  return cuda_status(rsk::launch_barrier_timeout_probe(h->s, as_stream(stream)));
}

int rs_check_acceptance(int mode, int64_t n, unsigned long long* count_dev, void* stream) {
  if (!count_dev || mode < 0 || mode > 1 || (mode == 1 && n < 1)) return RS_ERR_ARG;
  return cuda_status(rsk::launch_check_acceptance(mode, n, count_dev, as_stream(stream)));
}

int rs_check_weight_exp(double bound, unsigned long long* count_dev, double* max_rel_dev,
                        void* stream) {
  if (!count_dev || !max_rel_dev || !(bound > 0.0)) return RS_ERR_ARG;
  return cuda_status(rsk::launch_check_weight_exp(bound, count_dev, max_rel_dev, as_stream(stream)));
}

int rs_set_batched_launch(rs_handle* h, int kernel, int block, int items_per_thread) {
  if (!h || kernel < 0 || kernel >= rsk::kCfgCount) return RS_ERR_ARG;
  if (!valid_launch(block, items_per_thread)) return RS_ERR_ARG;
  h->s.batch_cfg[kernel] = rsk::LaunchCfg{block, items_per_thread};
  return RS_OK;
}

int rs_get_batched_launch(rs_handle* h, int kernel, int* block, int* items_per_thread) {
  if (!h || kernel < 0 || kernel >= rsk::kCfgCount || !block || !items_per_thread)
    return RS_ERR_ARG;
  *block = h->s.batch_cfg[kernel].block;
  *items_per_thread = h->s.batch_cfg[kernel].ipt;
  return RS_OK;
}

int rs_tune_batched(rs_handle* h, int dtype, const void* logw_dev, const int64_t* offsets_dev,
                    int32_t F, const int32_t* B_dev, int32_t B, int reps, void* stream) {
  if (!h || reps < 1 || reps > 1000) return RS_ERR_ARG;
  if (dtype != RS_F32 && dtype != RS_F64) return RS_ERR_ARG;
  const cudaStream_t s = as_stream(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return RS_ERR_ARG;  // timing needs real executions
  int st = set_device(h);
  if (st != RS_OK) return st;
  rsk::Scratch& sc = h->s;
  const int which = dtype == RS_F64 ? rsk::kCfgMetropolisF64 : rsk::kCfgMetropolisF32;
  const rsk::LaunchCfg saved_m = sc.batch_cfg[which], saved_p = sc.batch_cfg[rsk::kCfgPermute];
  // The caller's Metropolis call, its outputs in the handle's scratch: without Permute into
  // a_tmp (times the Metropolis kernel alone), with Permute into W (large enough for N int32).
  int32_t* spare = static_cast<int32_t*>(sc.W);
  auto run = [&](int permute) {
    return rs_resample_batched(h, RS_METROPOLIS, dtype, logw_dev, offsets_dev, F, B_dev, B, 0,
                               0, permute ? spare : sc.a_tmp, permute, nullptr, stream);
  };
  if ((st = run(0)) != RS_OK) return st;  // argument errors before any timing
  static const int kBlocks[] = {128, 256, 512};
  static const int kIpts[] = {1, 2, 4};
  for (int stage = 0; stage < 2; ++stage) {
    const int k = stage == 0 ? which : rsk::kCfgPermute;
    float best = -1.0f;
    rsk::LaunchCfg best_cfg = sc.batch_cfg[k];
    for (int b : kBlocks)
      for (int q : kIpts) {
        sc.batch_cfg[k] = rsk::LaunchCfg{b, q};
        const float ms = time_calls(s, reps, [&]() { return run(stage); });
        if (ms < 0.0f) {
          sc.batch_cfg[which] = saved_m;
          sc.batch_cfg[rsk::kCfgPermute] = saved_p;
          return RS_ERR_CUDA;
        }
        if (best < 0.0f || ms < best) {
          best = ms;
          best_cfg = sc.batch_cfg[k];
        }
      }
    sc.batch_cfg[k] = best_cfg;
  }
  return RS_OK;
}

int rs_capture_if_below(rs_handle* h, const double* value_dev, double threshold, void* stream,
                        void** body_stream) {
  if (!h || !value_dev || !body_stream || !stream || h->cap_active) return RS_ERR_ARG;
  int st = set_device(h);
  if (st != RS_OK) return st;
  const cudaStream_t s = as_stream(stream);
  cudaStreamCaptureStatus status = cudaStreamCaptureStatusNone;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edata = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(s, &status, nullptr, &graph, &deps, &edata, &nd) != cudaSuccess)
    return RS_ERR_CUDA;
  if (status != cudaStreamCaptureStatusActive) return RS_ERR_ARG;
  cudaGraphConditionalHandle hnd;
  if (cudaGraphConditionalHandleCreate(&hnd, graph, 0, cudaGraphCondAssignDefault) != cudaSuccess)
    return RS_ERR_CUDA;
  if (rsk::launch_set_if_below(hnd, value_dev, threshold, s) != cudaSuccess) return RS_ERR_CUDA;
  if (cudaStreamGetCaptureInfo(s, &status, nullptr, &graph, &deps, &edata, &nd) != cudaSuccess)
    return RS_ERR_CUDA;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = hnd;
  p.conditional.type = cudaGraphCondTypeIf;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, graph, deps, edata, nd, &p) != cudaSuccess) return RS_ERR_CUDA;
  if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                          cudaStreamSetCaptureDependencies) != cudaSuccess)
    return RS_ERR_CUDA;
  if (cudaStreamBeginCaptureToGraph(h->body_stream, p.conditional.phGraph_out[0], nullptr,
                                    nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return RS_ERR_CUDA;
  h->cap_active = true;
  h->cap_stream = s;
  h->saved_mode = h->s.launch_mode;
  h->s.launch_mode = RS_LAUNCH_SEPARATE;  // no cooperative launches inside the body
  rsk::pdl_disabled() = true;
  *body_stream = h->body_stream;
  return RS_OK;
}

int rs_capture_end_if(rs_handle* h, void* stream) {
  if (!h || !h->cap_active || as_stream(stream) != h->cap_stream) return RS_ERR_ARG;
  cudaGraph_t body = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->body_stream, &body);
  h->cap_active = false;
  h->s.launch_mode = h->saved_mode;
  rsk::pdl_disabled() = false;
  if (e != cudaSuccess) return RS_ERR_CUDA;
  // a plain kernel node after the conditional node: the next launch on the stream may carry a
  // programmatic dependency, which must follow a kernel
  return cuda_status(rsk::launch_noop(as_stream(stream)));
}

int rs_smc_mark_resampled(rs_handle* h, float* logw_dev, int64_t N, double* base_dev,
                          double log_n, int32_t* count_dev, void* stream) {
  if (!h || !logw_dev || !base_dev) return RS_ERR_ARG;
  int st = check_n(nullptr, N);
  if (st != RS_OK) return st;
  if ((st = set_device(h)) != RS_OK) return st;
  const cudaError_t e = rsk::launch_mark_resampled(h->s, logw_dev, N, base_dev, log_n, count_dev,
                                                   as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_smc_loglik_step(rs_handle* h, const double* lse_dev, double* base_dev, double* ll_dev,
                       int32_t* count_dev, double c, double log_n, int first, void* stream) {
  if (!h || !lse_dev || !base_dev || !ll_dev || (first != 0 && first != 1)) return RS_ERR_ARG;
  int st = set_device(h);
  if (st != RS_OK) return st;
  const cudaError_t e = rsk::launch_loglik_step(h->s, lse_dev, base_dev, ll_dev, count_dev, c,
                                                log_n, first, as_stream(stream));
  end_mark(h, as_stream(stream));
  return cuda_status(e);
}

int rs_metropolis_B(double eps, double beta, int32_t* B) {
  if (!B || !(eps > 0.0 && eps < 1.0) || !(beta > 0.0 && beta <= 1.0)) return RS_ERR_ARG;
  if (beta >= 1.0) {
    *B = 1;
    return RS_OK;
  }
  const double b = std::ceil(std::log(eps) / std::log1p(-beta));
  if (!(b <= 2147483647.0)) return RS_ERR_ARG;
  *B = b < 1.0 ? 1 : static_cast<int32_t>(b);
  return RS_OK;
}

int rs_last_error(rs_handle* h, void* stream) {
  if (!h) return RS_ERR_ARG;
  int st = set_device(h);
  if (st != RS_OK) return st;
  const cudaStream_t s = as_stream(stream);
  int v = rsk::kNoError;
  const int none = rsk::kNoError;
  if (cudaStreamSynchronize(s) != cudaSuccess) return RS_ERR_CUDA;
  if (cudaMemcpy(&v, h->s.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return RS_ERR_CUDA;
  if (cudaMemcpy(h->s.err, &none, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return RS_ERR_CUDA;
  if (v == -RS_ERR_TIMEOUT) {  // a grid barrier gave up: its arrival counter may be stale
    if (cudaMemset(&h->s.glob->bar.count, 0, sizeof(unsigned int)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
      return RS_ERR_CUDA;
  }
  return v == rsk::kNoError ? RS_OK : -v;
}

const char* rs_strerror(int status) {
  switch (status) {
    case RS_OK: return "ok";
    case RS_ERR_ARG: return "invalid argument or out-of-range index";
    case RS_ERR_NONFINITE: return "a log-weight is NaN or +inf";
    case RS_ERR_ZERO_WEIGHT: return "every weight is zero";
    case RS_ERR_BOUND_VIOLATED: return "rejection: a log-weight exceeds log_wmax";
    case RS_ERR_REJECTION_CAP: return "rejection: a particle reached max_trials";
    case RS_ERR_TIMEOUT: return "a bounded device wait gave up";
    case RS_ERR_CUDA: return "CUDA runtime error";
    case RS_ERR_CAPACITY: return "N exceeds the handle's max_n";
    default: return "unknown status";
  }
}

}  // extern "C"
