// rbo_gram_noalloc: the tall-skinny Gram C = X^T Y without any allocation.
//
// Some callers cannot let a library allocate device memory: applications whose
// HBM is already owned by another allocator (a framework that reserved the free
// memory for its own pool, where a cudaMalloc inside a library call fails or
// fragments that pool), code that must not trigger the device-wide
// synchronisation that cudaMalloc / cudaFree imply inside a latency-critical
// loop, and programs that fix their memory budget at start-up.  For them this
// entry point runs the same row-pass kernel as rbo_gram with its cross-CTA
// reduction scratch (partial sums, group partials, tickets, status word) in one
// file-scope __device__ array of RBO_NOALLOC_SCRATCH_BYTES, which every GPU that
// loads the library holds until the process exits.  The caller passes the inputs
// and a device array for the result.
//
// The array is shared by every call on a device and keeps the previous call's
// contents; each call clears the tickets and the status word it relies on.
// Calls that overlap on the GPU (other streams, other host threads) race on the
// array and must be serialised by the caller.
#include <mutex>

#include "rbo_internal.cuh"

namespace rbo {
namespace {

constexpr size_t kHeader = 1024;  // status word (64 B) + reduction tickets
static __device__ __align__(256) unsigned char g_noalloc_scratch[RBO_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once per
// device, with that device current, and cached (a cudaDeviceReset reloads the
// module and invalidates the cached address; the library is not used across one).
int scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return RBO_ERR_NO_DEVICE;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_ptr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return note_cuda(e != cudaSuccess ? e : cudaErrorUnknown);
    g_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_ptr[dev];
  return RBO_OK;
}

}  // namespace
}  // namespace rbo

extern "C" int rbo_gram_noalloc(int64_t n, int32_t a, const double* X, int64_t ldx, int32_t b,
                                const double* Y, int64_t ldy, double* C, void* stream) {
  using namespace rbo;
  if (n < 1 || a < 1 || a > 128 || b < 1 || b > 64 || !X || !Y || !C || ldx < n || ldy < n)
    return RBO_ERR_ARG;
  if ((int64_t)a * b > RBO_NOALLOC_MAX_AB) return RBO_ERR_ARG;
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RBO_ERR_NO_DEVICE;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return RBO_ERR_NO_DEVICE;
  unsigned char* base = nullptr;
  int e = scratch_address(&base);
  if (e) return e;
  cudaStream_t st = (cudaStream_t)stream;

  // An arena view of the static array: nothing can be taken from it (used == cap),
  // the reduction scratch is everything after the header.
  Arena ar;
  ar.device = dev;
  ar.base = reinterpret_cast<char*>(base);
  ar.cap = RBO_NOALLOC_SCRATCH_BYTES;
  ar.used = ar.cap;
  ar.status = reinterpret_cast<DevStatus*>(base);
  ar.tickets = reinterpret_cast<unsigned*>(base + 64);
  ar.n_tickets = (int)((kHeader - 64) / 4);
  ar.red = reinterpret_cast<double*>(base + kHeader);
  ar.red_bytes = RBO_NOALLOC_SCRATCH_BYTES - kHeader;

  // the grid is capped so that the per-CTA and per-group partials fit the array
  const int64_t L = (int64_t)a * b;
  const int64_t slots = (int64_t)(ar.red_bytes / 8) / L;     // partial vectors that fit
  int max_ctas = (int)std::min<int64_t>((slots * 16) / 17, 16 * (ar.n_tickets - 1));
  if (max_ctas < 1) return RBO_ERR_ARG;

  if ((e = note_cuda(cudaMemsetAsync(base, 0, kHeader, st)))) return e;
  RowPass r;
  r.n = n;
  r.X = X;
  r.ldx = ldx;
  r.a = a;
  r.Y = const_cast<double*>(Y);
  r.ldy = ldy;
  r.b = b;
  r.acc_x = 1;
  r.max_ctas = max_ctas;
  r.epi.op = EPI_STORE;
  r.epi.out = C;
  r.epi.out_ld = a;
  if ((e = rowpass_launch(r, &ar, st, nullptr))) return e;
  DevStatus hs;
  if ((e = note_cuda(cudaMemcpyAsync(&hs, base, sizeof(hs), cudaMemcpyDeviceToHost, st)))) return e;
  if ((e = note_cuda(cudaStreamSynchronize(st)))) return e;
  return hs.code;
}
