// noalloc.cu -- an allocation-free variant of the exact-SRE call (two-pass kernel, 16 <= N <= 20).
// The paper has no counterpart; this is a calling convenience.
//
// Some callers cannot allocate device memory at the point where they want this number:
//   * code running inside a host application or framework that owns all of the device's memory
//     through its own pool or a budget fixed at start-up, where an extra cudaMalloc either fails
//     or is not permitted;
//   * latency-critical loops that must not pay the implicit device-wide synchronisation of
//     cudaMalloc / cudaFree;
//   * plugins that must not change the process's device-memory footprint after they load.
// hadamag_sre_noalloc serves them: it needs no context and no caller scratch, and it calls no
// allocating routine.  Its scratch (the pass-1/pass-2 ring, the dependency counters, the status
// word and the per-CTA partial sums) lives in one file-scope __device__ array of fixed size
// (kBytes, 8.06 MiB), which every GPU that loads this library keeps until the process exits.
//
// Consequences a caller has to respect:
//   * The array is shared by every call on a device and keeps the last call's contents; each
//     call clears the counters and the status word it relies on.  Calls whose execution
//     overlaps on the GPU (different streams, or different host threads) race on the array:
//     serialise them.
//   * The first call on a device does the set-up: with that device current it looks up the
//     array's device address (cudaGetSymbolAddress) and caches it for the life of the process.
//     Make that first call before any stream capture.  The cached address does not survive
//     cudaDeviceReset: do not use this call on a device after resetting it.
#include <cmath>
#include <mutex>

#include "../../include/hadamag.h"
#include "sre_fwd.h"
#include "status_bits.h"

namespace hm {
namespace {

constexpr int kMinN = 16, kMaxN = 20;
constexpr size_t kRingBytes = (size_t)2 << (kMaxN + 2);   // 2 slots x 2^(N-1) complex64 at N = 20: 8 MiB
constexpr size_t kCounterOff = kRingBytes;                // 2 x 64 unsigned
constexpr size_t kStatusOff = kCounterOff + 512;          // int
constexpr size_t kResOff = kStatusOff + 256;              // 3 doubles
constexpr size_t kPartOff = kResOff + 256;                // per-CTA triples
constexpr int kMaxGrid = 2048;
constexpr size_t kBytes = kPartOff + (size_t)kMaxGrid * 3 * sizeof(double);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kBytes];

std::mutex g_lock;
void* g_addr[128] = {nullptr};

// Host-side address of the array on the current device (looked up once per device).
cudaError_t scratch_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lk(g_lock);
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return cudaSuccess;
}

// out[0] = M_n (NaN if a device check failed), out[1] = lost_norm, out[2] = device status bits.
__global__ void noalloc_finish(const double* __restrict__ res, const int* __restrict__ status, int N, double n,
                               double* __restrict__ out) {
    const double two_n = ldexp(1.0, N);
    double M;
    if (n == 1.0) M = -res[2] / res[1] + log2(res[1]) - (double)N;
    else M = log2(res[0] / two_n) / (1.0 - n);
    const int st = *status;
    out[0] = st ? nan("") : (M == 0.0 ? 0.0 : M);
    out[1] = 1.0 - res[1] / two_n;
    out[2] = (double)st;
}

}  // namespace
}  // namespace hm

extern "C" hadamag_status hadamag_sre_noalloc(const void* psi_dev, int N, double n, double* out_dev,
                                              hadamag_stream_t stream) {
    using namespace hm;
    if (!psi_dev || ((uintptr_t)psi_dev & 15u) || !out_dev || ((uintptr_t)out_dev & 7u))
        return HADAMAG_ERR_INVALID_ARG;
    if (!(n > 0.0) || !std::isfinite(n)) return HADAMAG_ERR_INVALID_ARG;
    if (N < kMinN || N > kMaxN) return HADAMAG_ERR_UNSUPPORTED;  // outside what the fixed array holds
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HADAMAG_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HADAMAG_ERR_CUDA;
    unsigned char* base = nullptr;
    if (scratch_address(dev, &base) != cudaSuccess) return HADAMAG_ERR_CUDA;

    const int mode = n == 1.0 ? 1 : n == 2.0 ? 2 : n == 3.0 ? 3 : 0;
    const int M = N - 11;  // pass-1 width 10 for N <= 20
    TwoPassParams P{};
    P.psi = reinterpret_cast<const float2*>(psi_dev);
    P.N = N;
    P.nq = n;
    P.count = int64_t(1) << N;
    P.a_list = nullptr;
    P.scratch = reinterpret_cast<float2*>(base);
    P.R = 2;  // two slots: the smallest ring the task order allows
    P.A = 1;
    P.U = 8;
    P.UPW = 2;
    P.TPT = 2;
    P.lag = 1;
    P.a_base = 0;
    P.n_batches = P.count;
    P.p1 = (1 << M) / (P.U * P.UPW);
    P.p2 = twopass_tiles_per_a(N) / P.TPT;
    P.done1 = reinterpret_cast<unsigned*>(base + kCounterOff);
    P.done2 = P.done1 + 64;
    P.status = reinterpret_cast<int*>(base + kStatusOff);
    P.spin_limit = kDefaultSpinLimit;
    P.wait_bias = 0;
    P.out = reinterpret_cast<double*>(base + kPartOff);
    P.per_a = 0;
    int grid = 0;
    if (twopass_max_grid(N, mode, sms, &grid) != cudaSuccess) return HADAMAG_ERR_CUDA;
    if (grid > kMaxGrid) grid = kMaxGrid;
    // counters and status must start at zero; the array keeps whatever the last call left
    if (cudaMemsetAsync(base + kCounterOff, 0, kResOff - kCounterOff, st) != cudaSuccess) return HADAMAG_ERR_CUDA;
    if (launch_twopass(P, mode, grid, st) != cudaSuccess) return HADAMAG_ERR_CUDA;
    double* res = reinterpret_cast<double*>(base + kResOff);
    if (launch_sum_triples(P.out, grid, res, st) != cudaSuccess) return HADAMAG_ERR_CUDA;
    noalloc_finish<<<1, 1, 0, st>>>(res, P.status, N, n, out_dev);
    if (cudaGetLastError() != cudaSuccess) return HADAMAG_ERR_CUDA;
    return HADAMAG_OK;
}
