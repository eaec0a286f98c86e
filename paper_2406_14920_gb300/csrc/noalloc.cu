// J/K build for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need J and K:
// code running while a CUDA graph is being captured, code inside a memory
// pool or allocator that must not re-enter the allocator, and real-time or
// embedded hosts that forbid allocation after start-up.  eri_build_jk itself
// allocates nothing once its plan exists, but it works in buffers the plan
// allocated.  This entry point instead takes its scratch from one fixed array
// that is part of the loaded library, so a build allocates nothing at all
// beyond what the caller passes in.
#include <atomic>
#include <cstdio>

#include "../../include/eri.h"
#include "plan.cuh"

int eri_build_jk_scratch(eri_plan_t* plan, const double* D, double* J, double* K, double* Dp, double* Kh, double* Jh,
                         cudaStream_t s);
int eri_plan_nbf_device(eri_plan_t* plan, int* nbf, int* device, int* nmol);

// Scratch: scaled density D', half-K and half-J accumulators, each nbf x nbf
// doubles, for nbf <= ERI_NOALLOC_MAX_NBF: 3 * 256 * 256 * 8 B = 1.5 MiB held by
// every GPU that loads this library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[3 * ERI_NOALLOC_MAX_NBF * ERI_NOALLOC_MAX_NBF];

static constexpr int kMaxDevices = 64;
static std::atomic<double*> g_scratch_dev[kMaxDevices] = {};

// Device address of the scratch array on `device` (must be current).  The host
// symbol g_noalloc_scratch is only a stand-in, never a device address, so it is
// looked up once per device with cudaGetSymbolAddress and cached.  Two threads
// making their first call at once both look it up and store the same address
// (atomic stores, no torn value).  cudaDeviceReset ends the context the address
// belongs to, and the cache cannot see that: a process that resets a device
// must not call eri_build_jk_noalloc on it again.
static int scratch_for(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return ERI_EUNSUPPORTED;
  double* p = g_scratch_dev[device].load(std::memory_order_acquire);
  if (!p) {
    void* q = nullptr;
    if (cudaGetSymbolAddress(&q, g_noalloc_scratch) != cudaSuccess || !q) return ERI_ECUDA;
    p = static_cast<double*>(q);
    g_scratch_dev[device].store(p, std::memory_order_release);
  }
  *out = p;
  return ERI_OK;
}

extern "C" int eri_build_jk_noalloc(eri_plan_t* plan, const double* D, double* J, double* K, void* stream) {
  if (!plan || !D || (!J && !K)) return ERI_EINVAL;
  int nbf = 0, device = 0, nmol = 1;
  eri_plan_nbf_device(plan, &nbf, &device, &nmol);
  if (nmol != 1) return ERI_EUNSUPPORTED;
  if (nbf > ERI_NOALLOC_MAX_NBF) {
    fprintf(stderr, "eri_build_jk_noalloc: %d basis functions exceed the fixed scratch limit of %d\n", nbf,
            ERI_NOALLOC_MAX_NBF);
    return ERI_EUNSUPPORTED;
  }
  if (cudaSetDevice(device) != cudaSuccess) return ERI_ECUDA;
  double* base = nullptr;
  int rc = scratch_for(device, &base);
  if (rc != ERI_OK) return rc;
  const size_t nn = (size_t)nbf * nbf;
  return eri_build_jk_scratch(plan, D, J, K, base, base + nn, base + 2 * nn, (cudaStream_t)stream);
}
