// pmmm_bin_sort_static: binning and stable sort of the particles by cell, with
// no device allocation at all.
//
// Some callers cannot call cudaMalloc: a host framework or memory pool that owns
// all device memory and forbids allocations behind its back, or a real-time
// loop that must never block in the allocator (cudaMalloc may synchronise the
// device and take an unbounded time).  They still get the first step of the
// force evaluation -- the cell ids, the stable permutation and the cell offsets
// -- through this entry point.  Its scratch (key and index double buffers,
// particle records, radix histograms, the error flag) is one file-scope device
// array, so the caller only passes the input and output buffers.
//
// The array is resident on every device that loads this library until the
// process exits.  Its device address is looked up once per device (with that
// device current) on the first call there; make that first call before any
// stream capture.  Every call waits for its stream to finish, because it reads
// the device-side status back.  Every call shares the array and it keeps the
// last call's contents: the error flag is cleared at the start of each call and
// everything else is fully rewritten before it is read.  Calls that overlap on
// the GPU (other streams, other host threads) race on the array and must not be
// made.
#include <mutex>

#include "internal.cuh"

using namespace pmmm;

namespace {

constexpr int64_t kMaxN = PMMM_STATIC_SORT_MAX_N;
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
// layout of the scratch array
constexpr size_t kKeys = align_up(sizeof(uint32_t) * kMaxN);                  // one key or index buffer
constexpr size_t kRec = align_up(4 * sizeof(double) * kMaxN);                 // particle records (FP64 size)
constexpr size_t kHist = align_up(sizeof(uint32_t) * 256 * ((kMaxN + 2047) / 2048));
constexpr size_t kChunks = align_up(sizeof(uint32_t) * 64);
constexpr size_t kErr = align_up(sizeof(int));
constexpr size_t kScratchBytes = 4 * kKeys + kRec + kHist + kChunks + kErr;

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};  // device address of g_sort_scratch, per device

// Device address of the scratch array on the current device (set-up on first use).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PMMM_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    // the host-side symbol is only a stand-in: the kernels need this device address
    if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return PMMM_ERR_CUDA;
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return PMMM_OK;
}

// any positive cell count per axis (the sort itself has no power-of-two rule)
bool mesh_dim_ok(int v) { return v >= 1; }

}  // namespace

extern "C" int pmmm_bin_sort_static(const pmmm_config* cfg, int64_t n, const void* pos, int32_t* perm,
                                    int32_t* cell_start, void* cuda_stream) {
  if (!cfg || n < 0 || !cell_start || (n > 0 && (!pos || !perm))) return PMMM_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a) {
    if (!(cfg->box_len[a] > 0.0) || !isfinite(cfg->box_len[a]) || !isfinite(cfg->box_lo[a])) return PMMM_ERR_INVALID_ARG;
    if (!mesh_dim_ok(cfg->mesh[a])) return PMMM_ERR_INVALID_ARG;
  }
  if (cfg->boundary != PMMM_OPEN && cfg->boundary != PMMM_PERIODIC) return PMMM_ERR_INVALID_ARG;
  if (cfg->precision < PMMM_FP64 || cfg->precision > PMMM_FP32_SPLITBF16_M2L) return PMMM_ERR_INVALID_ARG;
  const int64_t K = (int64_t)cfg->mesh[0] * cfg->mesh[1] * cfg->mesh[2];
  if (n > kMaxN || K > ((int64_t)1 << 28)) return PMMM_ERR_UNSUPPORTED;  // beyond the static workspace
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != PMMM_OK) return rc;
  unsigned char* b = (unsigned char*)base;
  SortWork w{};
  w.keys0 = (uint32_t*)(b);
  w.keys1 = (uint32_t*)(b + kKeys);
  w.vals0 = (uint32_t*)(b + 2 * kKeys);
  w.vals1 = (uint32_t*)(b + 3 * kKeys);
  void* rec = b + 4 * kKeys;
  w.hist = (uint32_t*)(b + 4 * kKeys + kRec);
  w.chunks = (uint32_t*)(b + 4 * kKeys + kRec + kHist);
  int* err = (int*)(b + 4 * kKeys + kRec + kHist + kChunks);
  w.cap = kMaxN;

  // geometry exactly as a plan derives it (the cell ids depend on lo, len and n / len)
  const Geo g = binning_geo(*cfg);
  const bool fp64 = cfg->precision == PMMM_FP64;

  cudaStream_t s = (cudaStream_t)cuda_stream;
  int nl = 0;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
  int key_bits = 0;
  while (((int64_t)1 << key_bits) < K) ++key_bits;
  uint32_t *keys_sorted = w.keys0, *vals_sorted = w.vals0;
  // the particle records written by the binning kernel are not used here; its
  // charge argument points at the positions so that every read stays in bounds
  if (e == cudaSuccess) e = launch_bin(pos, pos, fp64, n, g, w.keys0, rec, err, s, &nl);
  if (e == cudaSuccess) e = launch_radix_sort(w, n, key_bits, &keys_sorted, &vals_sorted, s, &nl);
  if (e == cudaSuccess) e = launch_cell_bounds(keys_sorted, n, K, cell_start, s, &nl);
  if (e == cudaSuccess && n > 0)
    e = cudaMemcpyAsync(perm, vals_sorted, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? PMMM_ERR_OOM : PMMM_ERR_CUDA;
  if (h & ERRBIT_NONFINITE) return PMMM_ERR_NONFINITE_INPUT;
  if (h & ERRBIT_OUT_OF_BOX) return PMMM_ERR_OUT_OF_BOX;
  return PMMM_OK;
}
