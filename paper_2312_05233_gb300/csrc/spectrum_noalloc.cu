// tnep_spectrum_noalloc: the spectrum tail without any device allocation.
//
// Some callers cannot call cudaMalloc: an MD engine that reserves all device
// memory for its own arena at start-up, or one that computes spectra inside
// its time-step loop, where cudaMalloc / cudaFree would add a device-wide
// synchronisation.  This entry point takes device buffers for the input and
// the outputs and keeps its scratch (the prepared signal, the
// autocorrelation and the cosine table) in the file-scope array below, which
// every GPU that loads the library holds until the process exits.

#include <mutex>

#include "tnep_internal.cuh"

namespace {

constexpr int kNoallocMaxT = TNEP_NOALLOC_MAX_T;
// signal [T][9] + acf [M+1] + cosine table [2M], with M < T
constexpr size_t kNoallocWords = (size_t)kNoallocMaxT * 9 + (size_t)kNoallocMaxT + 2 * (size_t)kNoallocMaxT;

static __device__ __align__(256) double g_spectrum_scratch[kNoallocWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

tnep_status noalloc_fail(tnep_status s, const char* msg) {
  tnep::set_last_error(msg);
  return s;
}

// True for device memory of device `dev` and for managed memory.  Device
// memory of another GPU is refused: the kernels run on the current device
// and would reach it through a peer address, which faults without peer access.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" tnep_status tnep_spectrum_noalloc(const double* series, int T, int C, double dt_fs, int kind,
                                             int max_lag, int subtract_mean, double* freq_cm1, double* spec,
                                             double* acf_out, void* stream) {
  if (!series || !freq_cm1 || !spec) return noalloc_fail(TNEP_ERR_INVALID, "NULL buffer");
  if (T < 2) return noalloc_fail(TNEP_ERR_INVALID, "need at least two samples");
  if (T > kNoallocMaxT)
    return noalloc_fail(TNEP_ERR_INVALID, "series longer than TNEP_NOALLOC_MAX_T (32768) samples");
  if (!(dt_fs > 0.0)) return noalloc_fail(TNEP_ERR_INVALID, "dt must be positive");
  if (kind == TNEP_SPECTRUM_IR) {
    if (C != 3) return noalloc_fail(TNEP_ERR_INVALID, "IR needs C = 3");
  } else if (kind == TNEP_SPECTRUM_RAMAN_ISO || kind == TNEP_SPECTRUM_RAMAN_ANISO) {
    if (C != 9) return noalloc_fail(TNEP_ERR_INVALID, "Raman needs C = 9");
  } else {
    return noalloc_fail(TNEP_ERR_INVALID, "unknown spectrum kind");
  }
  const int M = max_lag <= 0 ? T / 2 : max_lag;
  if (M < 1 || M >= T) return noalloc_fail(TNEP_ERR_INVALID, "max_lag must be in [1, T)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return noalloc_fail(TNEP_ERR_NO_DEVICE, "no current CUDA device");
  }
  if (!on_device(series, dev) || !on_device(freq_cm1, dev) || !on_device(spec, dev) ||
      (acf_out && !on_device(acf_out, dev)))
    return noalloc_fail(TNEP_ERR_INVALID, "series and outputs must be memory of the current device");
  double* scratch = nullptr;
  {
    // Set-up once per device, with that device current: the host-side name
    // of the array is not a device address, so ask the runtime for it.
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_spectrum_scratch);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(TNEP_ERR_CUDA, cudaGetErrorString(e));
      }
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // Every scratch element the kernels read is written earlier in the same
  // call, so nothing left by the previous call needs clearing.
  cudaError_t e = tnep::launch_spectrum(series, T, C, dt_fs, kind, M, subtract_mean, scratch, freq_cm1, spec,
                                        acf_out, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(TNEP_ERR_CUDA, cudaGetErrorString(e));
  }
  return TNEP_OK;
}
