// vf_poisson_solve_noalloc: the FFT Poisson solve of vf_poisson_solve for callers that cannot allocate device
// memory (for example code running where cudaMalloc is forbidden or unavailable: inside a host allocator hook,
// inside a framework that owns every device allocation, or a process that has pre-reserved all of its memory).
//
// Its scratch (the half spectrum and the FFT / eigenvalue tables) lives in one file-scope device array of
// kNoallocScratchBytes that every GPU which loads this library keeps until the process exits.  The array's name
// in host code is only a host-side stand-in, so its device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.  All calls share the array: calls that overlap on the GPU (two
// streams, two threads) race on it.  Nothing here needs zeroed scratch: the forward x pass writes every spectrum
// entry before any later pass reads it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "vf_internal.h"

namespace {

constexpr size_t kTableBytes = 1u << 20;                          // twiddle + eigenvalue tables
constexpr size_t kSpectrumBytes = 32u << 20;                      // half spectrum: nx*ny*nz values of T
constexpr size_t kNoallocScratchBytes = kTableBytes + kSpectrumBytes;
constexpr int kMaxAxis = 1024;                                    // longest table (nx/2 + 1, ny, nz)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up on the first successful call for that
// device.  Only a successful lookup is kept: a failed one (for example a first call made during stream capture)
// is tried again by the next call.
cudaError_t scratch_on_current_device(void** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();   // clear the lookup's error so the caller's next CUDA call does not see it
            return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Error return once work may be queued on st: wait for that work (its status is not needed) so that nothing of
// this call is still using the shared array when the caller's next call starts.
int drain_and_fail(cudaStream_t st)
{
    cudaStreamSynchronize(st);
    cudaGetLastError();
    return VF_ECUDA;
}

bool smooth235_even(int n)
{
    if (n < 8 || n % 2) return false;
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}

template <typename T>
int solve(int nx, int ny, int nz, double lx, double ly, double lz, const void* f, void* p, cudaStream_t st)
{
    struct C2 { T x, y; };
    const int M = nx / 2;
    const size_t cells = (size_t)nx * ny * nz;
    if (cells * sizeof(T) > kSpectrumBytes) return VF_ESIZE;
    if (M + 1 > kMaxAxis || ny > kMaxAxis || nz > kMaxAxis) return VF_ESIZE;
    const size_t tb = sizeof(T) == 8 ? 8 : 16;
    const size_t nmax = (size_t)(ny > nz ? ny : nz);
    if ((3 * tb * nmax + nmax) * sizeof(C2) > 227 * 1024) return VF_ESIZE;

    void* base = nullptr;
    if (scratch_on_current_device(&base) != cudaSuccess || !base) return VF_ECUDA;
    unsigned char* tables = static_cast<unsigned char*>(base);
    void* spectrum = tables + kTableBytes;

    // tables in host memory on the stack (about 90 KB; no heap, no device allocation), copied into the scratch
    C2 tw[4][kMaxAxis];
    T lam[3][kMaxAxis];
    const int tw_len[4] = {M, ny, nz, M + 1}, tw_n[4] = {M, ny, nz, nx};
    for (int t = 0; t < 4; ++t)
        for (int m = 0; m < tw_len[t]; ++m) {
            const double a = 2.0 * M_PI * (double)m / (double)tw_n[t];
            tw[t][m].x = (T)std::cos(a);
            tw[t][m].y = (T)(-std::sin(a));
        }
    const int lam_len[3] = {M, ny, nz}, lam_n[3] = {nx, ny, nz};
    const double h[3] = {lx / nx, ly / ny, lz / nz};
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < lam_len[j]; ++k) {
            const double s = (k == 0 || 2 * k == lam_n[j]) ? 0.0 : std::sin(2.0 * M_PI * (double)k / lam_n[j]);
            lam[j][k] = (T)(s * s / (h[j] * h[j]));
        }
    // table layout in the scratch: four twiddle tables, then three eigenvalue tables, each kMaxAxis long
    C2* dtw = reinterpret_cast<C2*>(tables);
    T* dlam = reinterpret_cast<T*>(tables + 4 * kMaxAxis * sizeof(C2));
    static_assert(4 * kMaxAxis * sizeof(double) * 2 + 3 * kMaxAxis * sizeof(double) <= kTableBytes, "tables");
    for (int t = 0; t < 4; ++t)
        if (cudaMemcpyAsync(dtw + (size_t)t * kMaxAxis, tw[t], tw_len[t] * sizeof(C2), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
            return drain_and_fail(st);
    for (int j = 0; j < 3; ++j)
        if (cudaMemcpyAsync(dlam + (size_t)j * kMaxAxis, lam[j], lam_len[j] * sizeof(T), cudaMemcpyHostToDevice,
                            st) != cudaSuccess)
            return drain_and_fail(st);

    vf::PoissonArgs<T> a{};
    a.nx = nx; a.ny = ny; a.nz = nz; a.M = M;
    a.f = const_cast<T*>(static_cast<const T*>(f));   // only read: no correction runs without a mask
    a.p = static_cast<T*>(p);
    a.smask = nullptr;
    a.n_near = 0;
    a.plane_layout = 0;
    a.spec = spectrum;
    a.twx = dtw;
    a.twy = dtw + kMaxAxis;
    a.twz = dtw + 2 * kMaxAxis;
    a.twr = dtw + 3 * kMaxAxis;
    a.lamx = dlam;
    a.lamy = dlam + kMaxAxis;
    a.lamz = dlam + 2 * kMaxAxis;
    for (int j = 0; j < 3; ++j) a.i2h2[j] = (T)(1.0 / (4.0 * h[j] * h[j]));
    a.invN = (T)(1.0 / (double)cells);
    a.ax = vf::make_fft_axis(M);
    a.ay = vf::make_fft_axis(ny);
    a.az = vf::make_fft_axis(nz);
    a.ny_div = vf::make_fast_div((uint32_t)ny);
    a.nx_div = vf::make_fast_div((uint32_t)nx);
    const int per_cta = sizeof(T) == 8 ? 1024 : 2048;   // complex values per CTA in the x passes
    a.rows_per_block = per_cta / M > 0 ? per_cta / M : 1;
    a.cols_per_block = (int)tb;
    if (vf::Kernels<T>::poisson_prepare(a) != cudaSuccess) return drain_and_fail(st);
    if (vf::Kernels<T>::poisson_iteration(a, 1, st) != cudaSuccess) return drain_and_fail(st);
    // the stack tables must stay alive until their copies have been consumed
    if (cudaStreamSynchronize(st) != cudaSuccess) return VF_ECUDA;
    return VF_OK;
}

}  // namespace

extern "C" int vf_poisson_solve_noalloc(int32_t nx, int32_t ny, int32_t nz, double lx, double ly, double lz,
                                        int32_t precision, const void* f, void* p, void* stream)
{
    if (!f || !p) return VF_EINVAL;
    if (!smooth235_even(nx) || !smooth235_even(ny) || !smooth235_even(nz)) return VF_ESIZE;
    if (!(lx > 0) || !(ly > 0) || !(lz > 0)) return VF_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (precision == VF_FP64) return solve<double>(nx, ny, nz, lx, ly, lz, f, p, st);
    if (precision == VF_FP32_MIXED) return solve<float>(nx, ny, nz, lx, ly, lz, f, p, st);
    return VF_EINVAL;
}

extern "C" int64_t vf_poisson_noalloc_max_cells(int32_t precision)
{
    if (precision == VF_FP64) return (int64_t)(kSpectrumBytes / sizeof(double));
    if (precision == VF_FP32_MIXED) return (int64_t)(kSpectrumBytes / sizeof(float));
    return 0;
}
