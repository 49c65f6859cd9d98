// Lagrangian particles (Sec. 2.3): one-way coupled, drag and gravity, implicit Euler.
//
//   du_p/dt = (C_d / tau_p)(u_f - u_p) + g,  tau_p = rho_p d^2 / (18 rho_f nu),  Re_p = |u_f - u_p| d / nu,
//   C_d = 1 + Re_p^(2/3) / 6,  dx_p/dt = u_p.
//
// One thread per particle, after the flow step: u_f is the new fluid velocity interpolated trilinearly between
// the eight cell centres (i h, periodic) around x_p; the drag coefficient is taken from the relative velocity at the
// start of the step, which makes the drag linear in the new velocity, u_p' = (u_p + a u_f + dt g) / (1 + a) with
// a = dt C_d / tau_p; then x_p' = x_p + dt u_p', wrapped into the box.  A particle whose new nearest cell is solid is
// deposited: it keeps its position, its velocity becomes 0 and it is not moved again.  Particle state is double
// (positions of metres resolved to far below a cell), the field is sampled in the grid's precision.
#include <cuda_runtime.h>

#include "vf_internal.h"

namespace vf {
namespace {

template <typename T>
__device__ __forceinline__ void load_uvw(const void* q, long long i, double out[3])
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

__device__ __forceinline__ long long wrapl(long long i, long long n) { i %= n; return i < 0 ? i + n : i; }

// fluid velocity at (x, y, z): weights of the eight surrounding cell centres, corners in z, y, x order
template <typename T>
__device__ void sample(const ParticleArgs& P, const void* q, const double pos[3], double uf[3])
{
    long long lo[3];
    double fr[3];
    const long long dims[3] = {P.nx, P.ny, P.nz};
    for (int j = 0; j < 3; ++j) {
        const double s = pos[j] / P.h[j];
        const double i0 = floor(s);
        fr[j] = s - i0;
        lo[j] = wrapl((long long)i0, dims[j]);
    }
    uf[0] = uf[1] = uf[2] = 0.0;
    for (int cz = 0; cz < 2; ++cz) {
        const double wz = cz ? fr[2] : 1.0 - fr[2];
        const long long iz = (lo[2] + cz) % dims[2];
        for (int cy = 0; cy < 2; ++cy) {
            const double wy = cy ? fr[1] : 1.0 - fr[1];
            const long long iy = (lo[1] + cy) % dims[1];
            for (int cx = 0; cx < 2; ++cx) {
                const double wx = cx ? fr[0] : 1.0 - fr[0];
                const long long ix = (lo[0] + cx) % dims[0];
                double v[3];
                load_uvw<T>(q, ix + dims[0] * (iy + dims[1] * iz), v);
                const double wgt = wx * wy * wz;
                for (int k = 0; k < 3; ++k) uf[k] += wgt * v[k];
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_particles(ParticleArgs P, const void* __restrict__ q,
                                                   const uint8_t* __restrict__ mask)
{
    const double dt = P.dyn ? P.dyn->dt : P.dt;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P.n;
         i += (long long)gridDim.x * blockDim.x) {
        if (P.state[i]) continue;
        const double pos[3] = {P.pos[0][i], P.pos[1][i], P.pos[2][i]};
        const double vel[3] = {P.vel[0][i], P.vel[1][i], P.vel[2][i]};
        const double d = P.size[i];
        double uf[3];
        sample<T>(P, q, pos, uf);
        double rel2 = 0.0;
        for (int k = 0; k < 3; ++k) rel2 += (uf[k] - vel[k]) * (uf[k] - vel[k]);
        const double re = sqrt(rel2) * d / P.nu;
        const double cd = 1.0 + pow(re, 2.0 / 3.0) / 6.0;
        const double tau = P.rho_p * d * d / (18.0 * P.rho_f * P.nu);
        const double a = dt * cd / tau;
        double nv[3], np[3];
        long long cell[3];
        const long long dims[3] = {P.nx, P.ny, P.nz};
        for (int k = 0; k < 3; ++k) {
            nv[k] = (vel[k] + a * uf[k] + dt * P.g[k]) / (1.0 + a);
            double x = fmod(pos[k] + dt * nv[k], P.L[k]);
            if (x < 0.0) x += P.L[k];
            np[k] = x;
            cell[k] = wrapl((long long)floor(x / P.h[k] + 0.5), dims[k]);
        }
        const long long c = cell[0] + dims[0] * (cell[1] + dims[1] * cell[2]);
        if (!(__ldg(mask + c) & kBitBeta)) {
            P.state[i] = 1;
            for (int k = 0; k < 3; ++k) P.vel[k][i] = 0.0;
            continue;
        }
        for (int k = 0; k < 3; ++k) {
            P.pos[k][i] = np[k];
            P.vel[k][i] = nv[k];
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
    k_particles<T><<<(unsigned)blocks, 256, 0, st>>>(P, q, mask);
    return cudaGetLastError();
}

template cudaError_t advance_particles<float>(const ParticleArgs&, const void*, const uint8_t*, cudaStream_t);
template cudaError_t advance_particles<double>(const ParticleArgs&, const void*, const uint8_t*, cudaStream_t);

}  // namespace vf
