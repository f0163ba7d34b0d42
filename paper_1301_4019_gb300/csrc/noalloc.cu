// noalloc.cu -- a systematic resampler that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs inside another framework's memory
// pool or allocator hooks, plugins whose host forbids device allocation after start-up,
// and real-time loops that must never block on the allocator. rs_systematic_noalloc serves
// them: it runs the same three kernels as rs_resample(RS_SYSTEMATIC, permute = 0), but its
// scratch (the status word, the per-CTA maxima and the per-tile sums and prefixes) lives in
// the file-scope device array below, which every GPU that loads this library holds until
// the process exits. The caller passes only inputs and outputs.
#include <cstddef>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace rsk {
namespace {

constexpr int64_t kNoAllocMaxN = RS_NOALLOC_MAX_N;
constexpr int64_t kNoAllocMaxTiles = (kNoAllocMaxN + kTile - 1) / kTile;
// Entries for the per-CTA maxima: the max pass runs 8 CTAs per SM, capped here (devices of
// up to 256 SMs get the full grid).
constexpr int kNoAllocMaxBlocks = 256 * 8;

// Layout of the static scratch (offsets in bytes, each 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }
constexpr size_t kOffGlob = 0;
constexpr size_t kOffErr = align256(kOffGlob + sizeof(ScanGlob));
constexpr size_t kOffBlockmax = align256(kOffErr + sizeof(int));
constexpr size_t kOffRec = align256(kOffBlockmax + sizeof(double) * kNoAllocMaxBlocks);
constexpr size_t kNoAllocBytes = align256(kOffRec + sizeof(double2) * 2 * seg_cap(kNoAllocMaxTiles));
static_assert(kNoAllocBytes <= 640 * 1024, "the static scratch must stay modest");

// Shared by every call on a device; zero at module load.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Resets the state that must start clean: the status word and the last-CTA counters.
__global__ void noalloc_begin_kernel() {
  pdl_wait();
  ScanGlob* g = reinterpret_cast<ScanGlob*>(g_noalloc_scratch + kOffGlob);
  g->ticket_max = 0u;
  g->ticket_tile = 0u;
  g->ticket_iscan = 0u;
  g->bar.count = 0u;
  g->bar.timeout_ns = kDefaultBarrierTimeoutNs;
  *reinterpret_cast<int*>(g_noalloc_scratch + kOffErr) = kNoError;
}

// Copies the call's device-side status to the caller's output word.
__global__ void noalloc_end_kernel(int32_t* status) {
  pdl_wait();
  const int v = *reinterpret_cast<const int*>(g_noalloc_scratch + kOffErr);
  *status = (v == kNoError) ? RS_OK : -v;
}

// Device addresses of g_noalloc_scratch, resolved once per device (host code only sees a
// host-side stand-in for the symbol, so the address must come from the runtime).
std::mutex g_setup_mutex;
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(unsigned char** out, cudaStream_t capture_check = nullptr,
                               bool check = false) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    // the lookup may load the module: not while the caller's stream is being captured
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (check && cudaStreamIsCapturing(capture_check, &cap) == cudaSuccess &&
        cap != cudaStreamCaptureStatusNone)
      return RS_ERR_ARG;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RS_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return RS_OK;
}

// A caller buffer must be device memory of the current device (or managed memory, which
// every device reaches): a pointer into another GPU's memory or into pageable host memory
// would make the kernels fault.
bool usable_here(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // the failed query leaves a (non-sticky) error: clear it
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

// Resolves the static array's address for the current device (rs_create calls it, so that a
// handle's device is ready for calls made during a stream capture).
int noalloc_prepare_current_device() {
  unsigned char* base = nullptr;
  return scratch_for_current_device(&base);
}

}  // namespace rsk

extern "C" int rs_systematic_noalloc(int dtype, const void* logw_dev, int64_t N, uint64_t seed,
                                     uint64_t step, int32_t* ancestors_dev, int32_t* status_dev,
                                     void* stream) {
  using namespace rsk;
  if (!logw_dev || !ancestors_dev) return RS_ERR_ARG;
  if (dtype != RS_F32 && dtype != RS_F64) return RS_ERR_ARG;
  if (N < 1) return RS_ERR_ARG;
  if (N > kNoAllocMaxN) return RS_ERR_CAPACITY;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return RS_ERR_CUDA;
  if (!usable_here(logw_dev, dev) || !usable_here(ancestors_dev, dev) ||
      (status_dev && !usable_here(status_dev, dev)))
    return RS_ERR_ARG;
  unsigned char* base = nullptr;
  const cudaStream_t cs = static_cast<cudaStream_t>(stream);
  const int st = scratch_for_current_device(&base, cs, true);
  if (st != RS_OK) return st;
  Scratch s;
  std::memset(&s, 0, sizeof(s));
  s.glob = reinterpret_cast<ScanGlob*>(base + kOffGlob);
  s.err = reinterpret_cast<int*>(base + kOffErr);
  s.blockmax = reinterpret_cast<double*>(base + kOffBlockmax);
  s.rec = reinterpret_cast<double2*>(base + kOffRec);
  s.max_n = kNoAllocMaxN;
  s.max_tiles = kNoAllocMaxTiles;
  s.max_blocks = device_sm_count() * 8 < kNoAllocMaxBlocks ? device_sm_count() * 8
                                                            : kNoAllocMaxBlocks;
  launch_pdl(noalloc_begin_kernel, 1, 1, cs);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = launch_scan_resample(s, RS_SYSTEMATIC, dtype == RS_F64 ? Acc::F64 : Acc::F32, logw_dev, N,
                             seed, step, 0u, ancestors_dev, nullptr, false, cs);
  if (e == cudaSuccess && status_dev) {
    launch_pdl(noalloc_end_kernel, 1, 1, cs, status_dev);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}
