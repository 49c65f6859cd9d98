// Internal interfaces between the C ABI / step engine (capi.cpp, host C++) and the CUDA kernels (*.cu).
// Only plain structs and host launchers appear here, so capi.cpp compiles with a host compiler.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime_api.h>

#include "../../include/ventflow.h"

namespace vf {

constexpr int kHistBins = 64;
constexpr int kMaxRadixStages = 16;

// Mask byte of a cell: bit 0 beta (fluid), bit 1 S (forcing region), bit 2 room region.
constexpr uint8_t kBitBeta = 1u;
constexpr uint8_t kBitS = 2u;
constexpr uint8_t kBitRoom = 4u;

// Constants of the flow kernels, in the compute precision T.
template <typename T>
struct FlowConsts {
    int nx, ny, nz;
    T i2h[3];     // 1 / (2 h_j)
    T i2h_div[3]; // 1 / (2 h_j dt): the divergence is stored divided by dt
    T i2h_dt[3];  // dt / (2 h_j): the pressure is stored as p / rho, the projection subtracts dt G p
    T q4h[3];     // 1 / (4 h_j): the 1/2 of the skew form times the 1/(2h) of the central difference
    T ih[3];      // 1 / h_j
    T ih2[3];     // 1 / h_j^2
    T nu, alpha, inv_tau;
    T dt6, dt3, dt2, dt;  // dt/6, dt/3, dt/2, dt
    T bf[3];      // body force
    T uset[3];    // forcing target velocity
    T cset;       // forcing target scalar
    T filt;       // pi^-6
};

// Pointers of one RK4 stage: q_s (stencil input), q_n, the accumulator and the output state.
template <typename T>
struct StageArgs {
    const T* qs[4];
    const T* qn[4];
    T* acc[4];
    T* out[4];
    const uint8_t* mask;
};

// One FFT axis: length and radix schedule (product of radix[] == n).
struct FftAxis {
    int n;
    int nstages;
    int radix[kMaxRadixStages];
};

// Everything one Poisson iteration needs.  The spectrum holds (nx/2) x ny x nz complex values, kx fastest;
// column kx = 0 packs the real spectra at kx = 0 (real part) and kx = nx/2 (imaginary part).
template <typename T>
struct PoissonArgs {
    int nx, ny, nz, M;        // M = nx / 2
    const T* r;               // right-hand side D u* (or the f of a plain solve)
    T* p;                     // in: p^k (for the (1 - beta) term), out: p^{k+1}
    const uint8_t* mask;
    int use_mask;             // 1: f = r + sum_j delta_j((1 - beta) delta_j p^k); 0: f = r
    void* spec;               // complex T [M * ny * nz]
    const void* twx;          // complex T [M]:  exp(-2 pi i m / M)
    const void* twy;          // complex T [ny]
    const void* twz;          // complex T [nz]
    const void* twr;          // complex T [M + 1]: exp(-2 pi i k / nx), real-FFT packing twiddles
    const T* lamx;            // [M]  sin^2(2 pi kx / nx) / hx^2 (kx = 0 and nx/2 share column 0, both 0)
    const T* lamy;            // [ny]
    const T* lamz;            // [nz]
    T i2h2[3];                // (1 / (2 h_j))^2
    T invN;                   // 1 / (nx ny nz)
    FftAxis ax, ay, az;
    int rows_per_block;       // rows of the x passes per CTA
    int cols_per_block;       // kx columns of the y / z passes per CTA
};

// Reduction scratch: per-CTA partial sums and histogram counts, and the output records.
struct ReduceArgsDev {
    double* partial;          // [nblocks * kRedSlots]
    int* hist_partial;        // [nblocks * (kHistBins + 2)]
    vf_reduce* out;           // single record (vf_reductions)
    vf_reduce* history;       // ring buffer
    long long* hist_count;    // records written so far
    long long* step_counter;  // device step counter
    int* nonfinite;           // set to 1 when a NaN / Inf is seen
    long long history_capacity;
    double dV;
    double dt;
    double t0;                // simulated time at step 0
};
constexpr int kRedSlots = 8;   // ke, div2, c_total, c_room, c2_room, v_room, div_max, u_max

// Called after each launch of a step when a step is profiled (pass = VF phase id, see vf_phase_name).
struct LaunchHook {
    void (*fn)(void* ctx, int phase);
    void* ctx;
    void operator()(int phase) const { if (fn) fn(ctx, phase); }
};

template <typename T>
struct Kernels {
    static cudaError_t stage(int s, const StageArgs<T>& a, const FlowConsts<T>& k, cudaStream_t st);
    static cudaError_t divergence(const T* u, const T* v, const T* w, T* r, const FlowConsts<T>& k,
                                  cudaStream_t st);
    // u = beta (u* - G p); ticks the device step counter.  c* is copied to out[3] when out[3] != cs.
    static cudaError_t project(const T* const us[3], const T* cs, const T* p, T* const out[4],
                               const uint8_t* mask, long long* step_counter, const FlowConsts<T>& k,
                               cudaStream_t st);
    static cudaError_t filter(const T* const in[4], T* const out[4], const uint8_t* mask, const FlowConsts<T>& k,
                              cudaStream_t st);
    static cudaError_t reduce(const T* const q[4], const uint8_t* mask, const FlowConsts<T>& k,
                              const ReduceArgsDev& r, int to_history, cudaStream_t st);
    static int reduce_blocks(const FlowConsts<T>& k);
    static cudaError_t poisson_prepare(const PoissonArgs<T>& a);   // shared-memory limits; call outside capture
    static cudaError_t poisson_iteration(const PoissonArgs<T>& a, cudaStream_t st, const LaunchHook* hook = nullptr);
    static cudaError_t convert_in(const void* src, int src_fp64, T* dst, size_t n, double scale,
                                  const uint8_t* mask, cudaStream_t st);
    static cudaError_t convert_out(const T* src, void* dst, int dst_fp64, size_t n, double scale,
                                   cudaStream_t st);
    static cudaError_t apply_mask(T* f, const uint8_t* mask, size_t n, cudaStream_t st);
    static size_t fft_smem_x(const PoissonArgs<T>& a);
    static size_t fft_smem_yz(const PoissonArgs<T>& a, int n);
};

// Mask helpers (precision independent).
cudaError_t mask_merge(uint8_t* mask, const uint8_t* src, uint8_t bit, size_t n, cudaStream_t st);
cudaError_t mask_fill(uint8_t* mask, uint8_t value, size_t n, cudaStream_t st);
cudaError_t mask_count_solid(const uint8_t* mask, size_t n, unsigned long long* d_count, cudaStream_t st);

}  // namespace vf
