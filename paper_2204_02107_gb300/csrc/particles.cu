// Lagrangian particles (Sec. 2.3): one-way coupled, drag and gravity, implicit Euler.
//
//   du_p/dt = (C_d / tau_p)(u_f - u_p) + g,  tau_p = rho_p d^2 / (18 rho_f nu),  Re_p = |u_f - u_p| d / nu,
//   C_d = 1 + Re_p^(2/3) / 6,  dx_p/dt = u_p.
//
// One thread per particle, after the flow step: u_f is the new fluid velocity interpolated trilinearly between
// the eight cell centres (i h, periodic) around x_p; the drag coefficient is taken from the relative velocity at the
// start of the step, which makes the drag linear in the new velocity, u_p' = (u_p + a u_f + dt g) / (1 + a) with
// a = dt C_d / tau_p; then x_p' = x_p + dt u_p', wrapped into the box.  A particle whose new nearest cell is solid is
// deposited: it keeps its position, its velocity becomes 0 and it is not moved again.  Particle state is stored
// in double; positions are accumulated in double (metres resolved to far below a cell), while the sampling and
// the drag run in the grid's precision (FP64 is a small fraction of FP32 throughput on this GPU).
#include <cuda_runtime.h>

#include "launch.cuh"
#include "vf_internal.h"

namespace vf {
namespace {

template <typename T>
__device__ __forceinline__ void load_uvw(const void* q, long long i, T out[3])
{
    if constexpr (sizeof(T) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(q) + i);
        out[0] = v.x; out[1] = v.y; out[2] = v.z;
    } else {
        const double2* p = reinterpret_cast<const double2*>(q) + 2 * i;
        const double2 a = __ldg(p), b = __ldg(p + 1);
        out[0] = a.x; out[1] = a.y; out[2] = b.x;
    }
}

// i modulo n in [0, n) for any i (also for the integer a NaN converts to): every index formed from a particle
// position stays inside the field, whatever the position holds
__device__ __forceinline__ int wrapi(long long i, int n)
{
    const long long r = i % n;
    return (int)(r < 0 ? r + n : r);
}

// coordinate / h: a division in double (as the oracle writes it), a multiplication by 1 / h in float
template <typename T>
__device__ __forceinline__ T scaled(double x, const ParticleArgs& P, int j)
{
    if constexpr (sizeof(T) == 8) return x / P.h[j];
    else return (T)x * (T)P.ih[j];
}

// fluid velocity at pos: weights of the eight surrounding cell centres, corners in z, y, x order
template <typename T>
__device__ void sample(const ParticleArgs& P, const void* q, const double pos[3], T uf[3])
{
    int lo[3];
    T fr[3];
    const int dims[3] = {P.nx, P.ny, P.nz};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const T s = scaled<T>(pos[j], P, j);
        const T i0 = floor(s);
        fr[j] = s - i0;
        lo[j] = wrapi((long long)i0, dims[j]);   // 0 <= pos < L, so i0 in [0, n]
    }
    uf[0] = uf[1] = uf[2] = T(0);
#pragma unroll
    for (int cz = 0; cz < 2; ++cz) {
        const T wz = cz ? fr[2] : T(1) - fr[2];
        const int iz = wrapi(lo[2] + cz, dims[2]);
#pragma unroll
        for (int cy = 0; cy < 2; ++cy) {
            const T wy = cy ? fr[1] : T(1) - fr[1];
            const int iy = wrapi(lo[1] + cy, dims[1]);
#pragma unroll
            for (int cx = 0; cx < 2; ++cx) {
                const T wx = cx ? fr[0] : T(1) - fr[0];
                const int ix = wrapi(lo[0] + cx, dims[0]);
                T v[3];
                load_uvw<T>(q, ix + (long long)dims[0] * (iy + (long long)dims[1] * iz), v);
                const T wgt = wx * wy * wz;
#pragma unroll
                for (int k = 0; k < 3; ++k) uf[k] += wgt * v[k];
            }
        }
    }
}

// Drag and gravity in the grid's precision T (the field's precision), positions accumulated in double.
template <typename T>
__global__ void __launch_bounds__(256) k_particles(ParticleArgs P, const void* __restrict__ q,
                                                   const uint8_t* __restrict__ mask)
{
    pdl_enter();
    const double dt = P.dyn ? P.dyn->dt : P.dt;
    const T dtt = (T)dt;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P.n;
         i += (long long)gridDim.x * blockDim.x) {
        if (P.state[i]) continue;
        const double pos[3] = {P.pos[0][i], P.pos[1][i], P.pos[2][i]};
        const T vel[3] = {(T)P.vel[0][i], (T)P.vel[1][i], (T)P.vel[2][i]};
        const T d = (T)P.size[i];
        T uf[3];
        sample<T>(P, q, pos, uf);
        T rel2 = T(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) rel2 += (uf[k] - vel[k]) * (uf[k] - vel[k]);
        const T re = sqrt(rel2) * d / (T)P.nu;
        const T r13 = cbrt(re);
        const T cd = T(1) + r13 * r13 / T(6);                     // 1 + Re^(2/3) / 6
        const T tau = (T)P.rho_p * d * d / (T(18) * (T)P.rho_f * (T)P.nu);
        const T a = dtt * cd / tau;
        T nv[3];
        double np[3];
        int cell[3];
        const int dims[3] = {P.nx, P.ny, P.nz};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            nv[k] = (vel[k] + a * uf[k] + dtt * (T)P.g[k]) / (T(1) + a);
            double x = pos[k] + dt * (double)nv[k];
            if (x < 0.0) x += P.L[k];                              // one box length covers any ordinary step
            else if (x >= P.L[k]) x -= P.L[k];
            if (!(x >= 0.0 && x < P.L[k])) {                       // a rounding below 0, a huge step, or NaN
                x = fmod(x, P.L[k]);
                if (x < 0.0) x += P.L[k];
                if (!(x >= 0.0 && x < P.L[k])) x = 0.0;
            }
            np[k] = x;
            cell[k] = wrapi((long long)floor((sizeof(T) == 8 ? x / P.h[k] : x * P.ih[k]) + 0.5), dims[k]);
        }
        const long long c = cell[0] + (long long)dims[0] * (cell[1] + (long long)dims[1] * cell[2]);
        if (!(__ldg(mask + c) & kBitBeta)) {
            P.state[i] = 1;
#pragma unroll
            for (int k = 0; k < 3; ++k) P.vel[k][i] = 0.0;
            continue;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            P.pos[k][i] = np[k];
            P.vel[k][i] = (double)nv[k];
        }
    }
}

}  // namespace

template <typename T>
cudaError_t advance_particles(const ParticleArgs& P, const void* q, const uint8_t* mask, cudaStream_t st)
{
    if (P.n <= 0) return cudaSuccess;
    long long blocks = (P.n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    return launch_pdl(k_particles<T>, dim3((unsigned)blocks), dim3(256), 0, st, P, q, mask);
}

template cudaError_t advance_particles<float>(const ParticleArgs&, const void*, const uint8_t*, cudaStream_t);
template cudaError_t advance_particles<double>(const ParticleArgs&, const void*, const uint8_t*, cudaStream_t);

}  // namespace vf
