// Flow kernels of the DNSLABIB time step (Sec. 2.1-2.2): fused RK4 stages, divergence, projection, sixth-order
// filter, FP64 reductions, and the small conversion / mask kernels behind the C ABI.
//
// Layout: the transported state (u, v, w, c) of a cell is one 4-vector (float4, or 32-byte aligned double4), so a
// stencil point of all four fields is one vector load; cells are ordered x fastest (index x + nx*(y + ny*z)),
// periodic in all three directions.  Pressure, divergence and mask are scalar arrays in the same order.  A CTA
// covers a 32 x 8 (x, y) tile and marches along z: the z neighbours stay in registers (the plane two ahead is
// prefetched one iteration early), the x and y neighbours come through L1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <type_traits>

#include "launch.cuh"
#include "vf_internal.h"

namespace vf {
namespace {

// Tile of a CTA (x by y threads).  Each CTA marches k.zc[kind] planes along z; the z-chunks are run-time
// parameters per kernel family (FlowConsts::zc), chosen by the autotuner or the defaults.
constexpr int TX = 32;
constexpr int TY = 8;
// rows of the filter's tile in FP32 (its shared-memory halo ring is 3 cells wide: the taller the tile, the fewer
// ring cells per filtered cell; 16 rows took 54.7 against 48.4 us per launch on the 256 x 128 x 128 room, the
// ring copies are not what bounds it); FP64 keeps TY within the static shared-memory limit
#ifndef VF_FILTER_TY
#define VF_FILTER_TY 8
#endif
template <typename T> __host__ __device__ constexpr int filter_ty() { return sizeof(T) == 4 ? VF_FILTER_TY : TY; }

__device__ __forceinline__ void ld4(const void* base, int i, float q[4])
{
    const float4 v = __ldg(reinterpret_cast<const float4*>(base) + i);
    q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
}
__device__ __forceinline__ void ld4(const void* base, int i, double q[4])
{
    const double2* p = reinterpret_cast<const double2*>(base) + 2 * (size_t)i;
    const double2 a = __ldg(p), b = __ldg(p + 1);
    q[0] = a.x; q[1] = a.y; q[2] = b.x; q[3] = b.y;
}
__device__ __forceinline__ void st4(void* base, int i, const float q[4])
{
    reinterpret_cast<float4*>(base)[i] = make_float4(q[0], q[1], q[2], q[3]);
}
__device__ __forceinline__ void st4(void* base, int i, const double q[4])
{
    double2* p = reinterpret_cast<double2*>(base) + 2 * (size_t)i;
    p[0] = make_double2(q[0], q[1]);
    p[1] = make_double2(q[2], q[3]);
}
// one component of a cell's 4-vector
template <typename T>
__device__ __forceinline__ T ld1(const void* base, int i, int comp)
{
    return __ldg(reinterpret_cast<const T*>(base) + 4 * (size_t)i + comp);
}

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <typename T>
__device__ __forceinline__ T beta_of(uint8_t m) { return (m & kBitBeta) ? T(1) : T(0); }

// Courant rate of one cell, sum_j |u_j| / h_j (Sec. 2.4 dynamic time step), with fixed rounding (no contraction)
// so that every kernel that forms it gets the same bits for the same velocity
__device__ __forceinline__ float sigma_cell(float u, float v, float w, const float ih[3])
{
    return __fadd_rn(__fadd_rn(__fmul_rn(fabsf(u), ih[0]), __fmul_rn(fabsf(v), ih[1])), __fmul_rn(fabsf(w), ih[2]));
}
__device__ __forceinline__ double sigma_cell(double u, double v, double w, const double ih[3])
{
    return __dadd_rn(__dadd_rn(__dmul_rn(fabs(u), ih[0]), __dmul_rn(fabs(v), ih[1])), __dmul_rn(fabs(w), ih[2]));
}

// CTA maximum of s, then one atomic max of its double bits per CTA (every thread of the CTA calls it; at most
// 32 warps)
__device__ __forceinline__ void sigma_flush(double s, unsigned long long* out)
{
    __shared__ double warp_max[32];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    if ((tid & 31) == 0) warp_max[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
        double m = warp_max[0];
        for (int w = 1; w < nw; ++w) m = fmax(m, warp_max[w]);
        if (m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
    }
}

// ------------------------------------------------------------------------------------------------------------
// RK4 stage: momentum and scalar right-hand sides and the stage combine (Sec. 2.1, Eqs. 2-4)
// ------------------------------------------------------------------------------------------------------------
// k_i = beta [ -sum_j q4h_j ((U_j Q_i)^+ - (U_j Q_i)^- + U_j^0 (Q_i^+ - Q_i^-))          (skew convection)
//              + nu sum_j ih2_j (Q_i^+ - 2 Q_i^0 + Q_i^-)                                  (diffusion)
//              + S (uset_i - Q_i^0) inv_tau + b_i ]                                        (forcing, body force)
// k_c = beta [ -sum_j ih_j (F^+ - F^-) + alpha sum_j ih2_j (beta^+ (c^+ - c^0) - beta^- (c^0 - c^-))
//              + S (cset - c^0) inv_tau ],  F^+ = beta^+ (U_j^0 c^0 + U_j^+ c^+) / 2 (face weight beta^0 beta^+,
//              beta^0 is applied by the outer factor)
// One cell of RK4 stage STAGE (the right-hand sides of Eqs. 2-3 above and the RK4 combine): from the centre q0, the
// axis neighbours qm[j], qp[j] (j = x, y, z), the cell's stencil mask sm (its beta and S, the neighbours' beta)
// and the cell's own q_n (stages 2-4) and q2, q3 (stage 4); leaves the stage output in o.
// FLUID: the cell and its six axis neighbours are fluid and the cell is outside the forcing region (sm is
// kSmFluid), so every beta factor is 1 and the forcing term is absent; the same bits as the general form, whose
// factors of 1 and forcing term of 0 change no value.
constexpr uint8_t kSmFluid = kSmSelf | kSmXm | kSmXp | kSmYm | kSmYp | kSmZm | kSmZp;

template <typename T, int STAGE, bool FLUID = false>
__device__ __forceinline__ void stage_cell(const StageArgs<T>& a, const FlowConsts<T>& k, int ic, const T q0[4],
                                           const T qm[3][4], const T qp[3][4], uint8_t sm, const T qn[4],
                                           const T q2[4], const T q3[4], T dt2, T dtf, T dt6, T inv_tau, T o[4])
{
    T bm[3], bp[3], beta = T(1), S = T(0);
    if constexpr (FLUID) {
#pragma unroll
        for (int j = 0; j < 3; ++j) bm[j] = bp[j] = T(1);
    } else {
        bm[0] = (sm & kSmXm) ? T(1) : T(0); bm[1] = (sm & kSmYm) ? T(1) : T(0); bm[2] = (sm & kSmZm) ? T(1) : T(0);
        bp[0] = (sm & kSmXp) ? T(1) : T(0); bp[1] = (sm & kSmYp) ? T(1) : T(0); bp[2] = (sm & kSmZp) ? T(1) : T(0);
        beta = (sm & kSmSelf) ? T(1) : T(0);
        S = (sm & kSmS) ? (a.sval ? __ldg(a.sval + ic) : T(1)) : T(0);
    }

    T kq[4];
    // velocity: the skew-symmetric term (U_j^+ Q_i^+ - U_j^- Q_i^-) + U_j^0 (Q_i^+ - Q_i^-) is grouped as
    // Q_i^+ (U_j^+ + U_j^0) - Q_i^- (U_j^- + U_j^0), the two sums shared by the three components, and the
    // Laplacian as sum_j ih2_j (Q_i^+ + Q_i^-) - (2 sum_j ih2_j) Q_i^0: the same sums in another rounding order
    T up[3], um[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        up[j] = qp[j][j] + q0[j];
        um[j] = qm[j][j] + q0[j];
    }
    const T ih2_2 = T(2) * (k.ih2[0] + k.ih2[1] + k.ih2[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T conv = T(0), diff = T(0);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            conv += k.q4h[j] * (qp[j][i] * up[j] - qm[j][i] * um[j]);
            diff += k.ih2[j] * (qp[j][i] + qm[j][i]);
        }
        diff -= ih2_2 * q0[i];
        if constexpr (FLUID) kq[i] = -conv + k.nu * diff + k.bf[i];
        else kq[i] = beta * (-conv + k.nu * diff + S * (k.uset[i] - q0[i]) * inv_tau + k.bf[i]);
    }
    {
        // the face fluxes' factor 1/2 is moved onto ih_j (a power-of-two scaling: the same bits)
        const T c0 = q0[3];
        T conv = T(0), diff = T(0);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const T uc0 = q0[j] * c0;
            if constexpr (FLUID) {
                const T Fp2 = uc0 + qp[j][j] * qp[j][3];
                const T Fm2 = qm[j][j] * qm[j][3] + uc0;
                conv += (T(0.5) * k.ih[j]) * (Fp2 - Fm2);
                diff += k.ih2[j] * ((qp[j][3] - c0) - (c0 - qm[j][3]));
            } else {
                const T Fp2 = bp[j] * (uc0 + qp[j][j] * qp[j][3]);
                const T Fm2 = bm[j] * (qm[j][j] * qm[j][3] + uc0);
                conv += (T(0.5) * k.ih[j]) * (Fp2 - Fm2);
                diff += k.ih2[j] * (bp[j] * (qp[j][3] - c0) - bm[j] * (c0 - qm[j][3]));
            }
        }
        if constexpr (FLUID) kq[3] = -conv + k.alpha * diff;
        else kq[3] = beta * (-conv + k.alpha * diff + S * (k.cset - c0) * inv_tau);
    }

    if (!FLUID && a.target && (sm & kSmS)) {
        // per-cell targets: the forcing above used targets of 0, add S beta target / tau_f
        T t4[4];
        ld4(a.target, ic, t4);
        const T sb = beta * S * inv_tau;
#pragma unroll
        for (int f = 0; f < 4; ++f) kq[f] += sb * t4[f];
    }

    // RK4 combine, classic tableau (nodes 0, 1/2, 1/2, 1; weights 1/6, 1/3, 1/3, 1/6) with the stage states as
    // the only registers: q2 = q_n + dt/2 k1, q3 = q_n + dt/2 k2, q4 = q_n + dt k3, so that
    // q* = q_n + dt/6 (k1 + 2 k2 + 2 k3 + k4) = (q2 + 2 q3 + q4 - q_n) / 3 + dt/6 k4  (q4 is the stencil centre)
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (STAGE == 1) o[f] = q0[f] + dt2 * kq[f];
        else if (STAGE == 2) o[f] = qn[f] + dt2 * kq[f];
        else if (STAGE == 3) o[f] = qn[f] + dtf * kq[f];
        else o[f] = (q2[f] + T(2) * q3[f] + q0[f] - qn[f]) * k.third + dt6 * kq[f];
    }
}

// ------------------------------------------------------------------------------------------------------------
// Scalar budget CTAs of the stage 3 and stage 4 launches (Eqs. 3-4 in flux form; the room inventory of Sec. 3.3).
// For every cell of the budget list and each of the launch's two stage states q_s (RK4 weight b_s): the relaxation
// source S (c_set - c_s) / tau_f of a fluid forcing cell (and again if the cell is in the room), and for a fluid
// room cell the flux of Eq. 3 through each face to a fluid neighbour outside the room -- convective
// (u_j c |_i + u_j c |_nb) / 2 minus diffusive alpha_c (c_nb - c_i) / h_j, counted out of the room -- times the face
// area dV / h_j.  A thread takes one (cell, state) item at a time and issues all of its loads (the cell's and its
// six neighbours' 4-vectors and mask bytes) before using them; the arithmetic is in double.  Each CTA leaves its
// partial sums; the last budget CTA of stage 4 (atomic ticket) adds both launches' partials in CTA order and
// scales by dt and dV.
// ------------------------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void ld4_cg(const void* base, size_t i, double q[4])
{
    if constexpr (sizeof(T) == 4) {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(base) + i);
        q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
    } else {
        const double2* p = reinterpret_cast<const double2*>(base) + 2 * i;
        const double2 a = __ldcg(p), b = __ldcg(p + 1);
        q[0] = a.x; q[1] = a.y; q[2] = b.x; q[3] = b.y;
    }
}

template <typename T, bool DYN>
__device__ __noinline__ void budget_cta(const StageArgs<T>& a, const FlowConsts<T>& k, int cta)
{
    const BudgetArgs& B = a.bud;
    const int nx = k.nx, ny = k.ny, nz = k.nz;
    const long long plane = (long long)nx * ny;
    const double inv_tau = DYN ? k.dyn->inv_tau : B.inv_tau;
    const int tid = threadIdx.x + TX * threadIdx.y;
    double f_all = 0.0, f_room = 0.0, outflow = 0.0;
    const long long items = 2LL * (B.n > 0 ? B.n : 0);
    for (long long j = (long long)cta * (TX * TY) + tid; j < items; j += (long long)B.ctas * (TX * TY)) {
        const long long i = B.list[j >> 1];
        const void* q = (j & 1) ? B.qb : B.qa;
        const double w = (j & 1) ? B.wb : B.wa;
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / plane);
        const long long nb[6] = {i - x + wrap(x - 1, nx), i - x + wrap(x + 1, nx),
                                 i + (long long)(wrap(y - 1, ny) - y) * nx, i + (long long)(wrap(y + 1, ny) - y) * nx,
                                 i + (long long)(wrap(z - 1, nz) - z) * plane,
                                 i + (long long)(wrap(z + 1, nz) - z) * plane};
        const uint8_t m = a.mask[i];
        uint8_t mn[6];
        double qc[4], qn[6][4];
        ld4_cg<T>(q, (size_t)i, qc);
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            mn[d] = a.mask[nb[d]];
            ld4_cg<T>(q, (size_t)nb[d], qn[d]);
        }
        if (!(m & kBitBeta)) continue;
        if (m & kBitS) {
            const double S = a.sval ? (double)a.sval[i] : 1.0;
            const double cset = a.target ? (double)__ldcg(reinterpret_cast<const T*>(a.target) + 4 * i + 3) : B.cset;
            const double f = w * (S * (cset - qc[3]) * inv_tau);
            f_all += f;
            if (m & kBitRoom) f_room += f;
        }
        if (m & kBitRoom) {
#pragma unroll
            for (int d = 0; d < 6; ++d) {
                if ((mn[d] & (kBitBeta | kBitRoom)) != kBitBeta) continue;   // a solid or room neighbour
                const int jx = d >> 1;
                const double sgn = (d & 1) ? 1.0 : -1.0;   // face at +h_j / 2 or -h_j / 2
                const double flux = sgn * 0.5 * (qc[jx] * qc[3] + qn[d][jx] * qn[d][3]) -
                                    B.alpha * (qn[d][3] - qc[3]) * B.ih[jx];
                outflow += w * flux * B.ih[jx];
            }
        }
    }
    __shared__ double wsum[kBudgetTerms][TX * TY / 32];
    __shared__ bool is_last;
    const int lane = tid & 31, wid = tid >> 5;
    double v[kBudgetTerms] = {f_all, f_room, outflow};
#pragma unroll
    for (int t = 0; t < kBudgetTerms; ++t) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[t] += __shfl_xor_sync(0xffffffffu, v[t], o);
        if (lane == 0) wsum[t][wid] = v[t];
    }
    __syncthreads();
    if (tid < kBudgetTerms) {
        double c = 0.0;
        for (int ww = 0; ww < TX * TY / 32; ++ww) c += wsum[tid][ww];
        B.partial[((size_t)B.slot * B.cap + cta) * kBudgetTerms + tid] = c;
    }
    if (B.slot == 0) return;
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(B.done, 1u) == (unsigned)(B.ctas - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (wid < kBudgetTerms) {
        double c = 0.0;
        for (int b = lane; b < B.ctas_prev; b += 32) c += __ldcg(B.partial + (size_t)b * kBudgetTerms + wid);
        for (int b = lane; b < B.ctas; b += 32)
            c += __ldcg(B.partial + ((size_t)B.cap + b) * kBudgetTerms + wid);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) {
            const double dt = DYN ? k.dyn->dt : B.dt;
            B.out[wid] = dt * B.dV * c;   // the outflow's face area dV / h_j: its 1 / h_j is already in c
        }
    }
    if (tid == 0) *B.done = 0u;
}

// Stage 4 reads three own states (q_n, q2, q3): prefetching them too takes 80 registers (3 CTAs per SM).
#ifndef VF_STAGE_PREFETCH_OWN4
#define VF_STAGE_PREFETCH_OWN4 0
#endif
constexpr bool kStagePrefetchOwn4 = VF_STAGE_PREFETCH_OWN4 != 0;

template <typename T, int STAGE, bool DYN>
__global__ void __launch_bounds__(TX * TY, sizeof(T) == 4 ? 4 : 1)
k_stage(StageArgs<T> a, FlowConsts<T> k)
{
    pdl_enter();
    int bz = blockIdx.z;
    if constexpr (STAGE >= 3) {
        if (a.bud.n >= 0) {   // the first z slice of the grid holds the budget CTAs
            if (bz == 0) {
                const int cta = blockIdx.x + gridDim.x * blockIdx.y;
                if (cta < a.bud.ctas) budget_cta<T, DYN>(a, k, cta);
                return;
            }
            --bz;
        }
    }
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= k.nx || y >= k.ny) return;
    const unsigned wmask = STAGE == 1 ? __activemask() : 0u;   // the warp's cells in the grid (same planes)
    // dt-dependent constants: kernel parameters for a fixed dt, the step's control block for a dynamic one
    T dt2 = k.dt2, dtf = k.dt, dt6 = k.dt6, inv_tau = k.inv_tau;
    if constexpr (DYN) {
        dt2 = (T)k.dyn->dt2;
        dtf = (T)k.dyn->dt;
        dt6 = (T)k.dyn->dt6;
        inv_tau = (T)k.dyn->inv_tau;
    }
    const int nx = k.nx, ny = k.ny, nz = k.nz;
    const int plane = nx * ny;
    const int zc = k.zc[kZcStage];
    const int z0 = bz * zc;
    const int z1 = min(z0 + zc, nz);
    const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
    const int rowc = y * nx, rowm = wrap(y - 1, ny) * nx, rowp = wrap(y + 1, ny) * nx;

    // z registers: the 4-vector at z-1, z, z+1 and the prefetched plane z+2; the stencil mask at z and z+1; the
    // cell's own q_n (and q2, q3 in stage 4) at z and, prefetched, at z+1 (stage 4 overwrites q2 with q* in place:
    // the cell at z+1 is read before its owner thread writes it).  The 4-vectors form a ring of 4 slots (plane
    // z + j - 1 in slot (P + j) mod 4 at phase P = (z - z0) mod 4) and the own states a ring of 2, so that with the
    // loop unrolled over the 4 phases every slot index is a constant and nothing is copied as the window moves.
    T Q[4][4] = {};
    T own[2][3][4] = {};   // q_n, q2, q3 of the cell at z (slot P mod 2) and z+1
    constexpr int NOWN = STAGE == 1 ? 0 : (STAGE == 4 ? 3 : 1);
    constexpr bool PF = STAGE != 4 || kStagePrefetchOwn4;   // prefetched one plane ahead, else read in place
    const void* own_src[3] = {a.qn, a.q2, a.q3};
    uint8_t m0, mzp;
    {
        const int im = wrap(z0 - 1, nz) * plane + rowc + x;
        const int ic = z0 * plane + rowc + x;
        const int ip = wrap(z0 + 1, nz) * plane + rowc + x;
        ld4(a.qs, im, Q[0]);
        ld4(a.qs, ic, Q[1]);
        ld4(a.qs, ip, Q[2]);
        m0 = __ldg(a.smask + ic);
        mzp = __ldg(a.smask + ip);
        if (PF) {
#pragma unroll
            for (int o = 0; o < NOWN; ++o) ld4(own_src[o], ic, own[0][o]);
        }
    }
    auto body = [&](auto phase, int z) {
        constexpr int P = decltype(phase)::value;
        constexpr int OC = PF ? P % 2 : 0, ON = PF ? (P + 1) % 2 : 0;   // own-state slots at z and z+1
        const int zb = z * plane;
        const int ic = zb + rowc + x;
        uint8_t mn2 = 0;
        if (z + 1 < z1) {   // prefetch plane z+2 of the stencil state and the cell's own states at z+1
            const int i2 = wrap(z + 2, nz) * plane + rowc + x;
            ld4(a.qs, i2, Q[(P + 3) % 4]);
            mn2 = __ldg(a.smask + i2);
            if (PF) {
#pragma unroll
                for (int o = 0; o < NOWN; ++o) ld4(own_src[o], ic + plane, own[ON][o]);
            }
        }
        if (!PF) {
#pragma unroll
            for (int o = 0; o < NOWN; ++o) ld4(own_src[o], ic, own[OC][o]);
        }
        T qm[3][4], qp[3][4];
        ld4(a.qs, zb + rowc + xm, qm[0]);
        ld4(a.qs, zb + rowc + xp, qp[0]);
        ld4(a.qs, zb + rowm + x, qm[1]);
        ld4(a.qs, zb + rowp + x, qp[1]);
#pragma unroll
        for (int f = 0; f < 4; ++f) { qm[2][f] = Q[P % 4][f]; qp[2][f] = Q[(P + 2) % 4][f]; }
        T o[4];
        // stage 1 (issue-bound) takes the fluid form where a warp, one row of 32 cells, is all fluid and away from
        // forcing (36.0 instead of 38.1 us on the 256 x 128 x 128 room); in stages 2-4 the second copy of the
        // arithmetic cost more than it saved (47.5 / 45.1 / 62.3 against 44.2 / 43.9 / 60.4 us)
        if (STAGE == 1 && __all_sync(wmask, m0 == kSmFluid))
            stage_cell<T, STAGE, true>(a, k, ic, Q[(P + 1) % 4], qm, qp, m0, own[OC][0], own[OC][1], own[OC][2],
                                       dt2, dtf, dt6, inv_tau, o);
        else
            stage_cell<T, STAGE>(a, k, ic, Q[(P + 1) % 4], qm, qp, m0, own[OC][0], own[OC][1], own[OC][2], dt2,
                                 dtf, dt6, inv_tau, o);
        st4(a.out, ic, o);
        m0 = mzp;
        mzp = mn2;
    };
    using I0 = std::integral_constant<int, 0>; using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>; using I3 = std::integral_constant<int, 3>;
    if constexpr (STAGE == 4) {
        // stage 4 holds three own states: unrolled, its loads of later planes are scheduled early and spill under
        // the 64-register bound, so its window moves by copies
        for (int z = z0; z < z1; ++z) {
            body(I0{}, z);
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int f = 0; f < 4; ++f) Q[j][f] = Q[j + 1][f];
        }
    } else {
        for (int z = z0; z < z1; z += 4) {
            body(I0{}, z);
            if (z + 1 >= z1) break;
            body(I1{}, z + 1);
            if (z + 2 >= z1) break;
            body(I2{}, z + 2);
            if (z + 3 >= z1) break;
            body(I3{}, z + 3);
        }
    }
}

// ------------------------------------------------------------------------------------------------------------
// Divergence r = sum_j delta_j u_j / dt (Eq. 9; divided by dt because the solver works on p / rho)
// ------------------------------------------------------------------------------------------------------------
constexpr int kDivGroup = 4;

template <typename T, bool DYN>
__global__ void __launch_bounds__(TX * TY) k_div(const void* __restrict__ q, T* __restrict__ r, FlowConsts<T> k)
{
    pdl_enter();
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= k.nx || y >= k.ny) return;
    T i2h[3] = {k.i2h_div[0], k.i2h_div[1], k.i2h_div[2]};
    if constexpr (DYN) {
#pragma unroll
        for (int j = 0; j < 3; ++j) i2h[j] = (T)k.dyn->i2h_div[j];
    }
    const int nx = k.nx, ny = k.ny, nz = k.nz;
    const int plane = nx * ny;
    const int z0 = blockIdx.z * k.zc[kZcDiv], z1 = min(z0 + k.zc[kZcDiv], nz);
    const int rowc = y * nx, rowm = wrap(y - 1, ny) * nx, rowp = wrap(y + 1, ny) * nx;
    const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
    // groups of kDivGroup planes, software-pipelined: the loads of the next group (its u and v neighbours and the w
    // of the planes above it) are issued before the current group is differenced, so two groups are in flight
    constexpr int U = kDivGroup;
    struct Group { T um[U], up[U], vm[U], vp[U], wz[U]; };   // wz[u]: w at plane z + u + 1
    auto load = [&](int zg, Group& g) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int z = zg + u;
            const bool ok = z < z1;
            const int zb = (ok ? z : z0) * plane;
            g.um[u] = ok ? ld1<T>(q, zb + rowc + xm, 0) : T(0);
            g.up[u] = ok ? ld1<T>(q, zb + rowc + xp, 0) : T(0);
            g.vm[u] = ok ? ld1<T>(q, zb + rowm + x, 1) : T(0);
            g.vp[u] = ok ? ld1<T>(q, zb + rowp + x, 1) : T(0);
            g.wz[u] = ok ? ld1<T>(q, wrap(z + 1, nz) * plane + rowc + x, 2) : T(0);
        }
    };
    T wzm = ld1<T>(q, wrap(z0 - 1, nz) * plane + rowc + x, 2);
    T wz0 = ld1<T>(q, z0 * plane + rowc + x, 2);
    Group cur, nxt;
    load(z0, cur);
    for (int zg = z0; zg < z1; zg += U) {
        if (zg + U < z1) load(zg + U, nxt);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int z = zg + u;
            if (z < z1) {
                const T wzp = cur.wz[u];
                const T d = i2h[0] * (cur.up[u] - cur.um[u]) + i2h[1] * (cur.vp[u] - cur.vm[u]) + i2h[2] * (wzp - wzm);
                r[z * plane + rowc + x] = d;
                wzm = wz0;
                wz0 = wzp;
            }
        }
        cur = nxt;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Projection u = beta (u* - dt G p) with p = p / rho (Eq. 8); c* passes through.  Ticks the device step counter.
// ------------------------------------------------------------------------------------------------------------
constexpr int kProjectGroup = 2;

template <typename T, bool DYN>
__global__ void __launch_bounds__(TX * TY) k_project(const void* __restrict__ qs, const T* __restrict__ p,
                                                     void* __restrict__ out, const uint8_t* __restrict__ mask,
                                                     long long* step_counter, FlowConsts<T> k,
                                                     unsigned long long* sigma_out)
{
    pdl_enter();
    if (step_counter && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
        threadIdx.y == 0)
        *step_counter += 1;
    T i2h[3] = {k.i2h_dt[0], k.i2h_dt[1], k.i2h_dt[2]};
    if constexpr (DYN) {
#pragma unroll
        for (int j = 0; j < 3; ++j) i2h[j] = (T)k.dyn->i2h_dt[j];
    }
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    T smax = T(0);   // Courant rate of the written velocity (DYN with the filter off: the step's final state)
    if (x < k.nx && y < k.ny) {
        const int nx = k.nx, ny = k.ny, nz = k.nz;
        const int plane = nx * ny;
        const int z0 = blockIdx.z * k.zc[kZcProject], z1 = min(z0 + k.zc[kZcProject], nz);
        const int rowc = y * nx, rowm = wrap(y - 1, ny) * nx, rowp = wrap(y + 1, ny) * nx;
        const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
        // groups of kProjectGroup planes, software-pipelined like the divergence: the next group's loads are in
        // flight while the current group is projected
        constexpr int U = kProjectGroup;
        struct Group { T q[U][4], pxm[U], pxp[U], pym[U], pyp[U], pz[U]; uint8_t m[U]; };   // pz[u]: p at z + u + 1
        auto load = [&](int zg, Group& g) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int z = zg + u;
                const bool ok = z < z1;
                const int zb = (ok ? z : z0) * plane;
                if (ok) {
                    ld4(qs, zb + rowc + x, g.q[u]);
                } else {
                    g.q[u][0] = g.q[u][1] = g.q[u][2] = g.q[u][3] = T(0);
                }
                g.m[u] = ok ? __ldg(mask + zb + rowc + x) : 0;
                g.pxm[u] = ok ? __ldg(p + zb + rowc + xm) : T(0);
                g.pxp[u] = ok ? __ldg(p + zb + rowc + xp) : T(0);
                g.pym[u] = ok ? __ldg(p + zb + rowm + x) : T(0);
                g.pyp[u] = ok ? __ldg(p + zb + rowp + x) : T(0);
                g.pz[u] = ok ? __ldg(p + wrap(z + 1, nz) * plane + rowc + x) : T(0);
            }
        };
        T pzm = __ldg(p + wrap(z0 - 1, nz) * plane + rowc + x);
        T pz0 = __ldg(p + z0 * plane + rowc + x);
        Group cur, nxt;
        load(z0, cur);
        for (int zg = z0; zg < z1; zg += U) {
            if (zg + U < z1) load(zg + U, nxt);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int z = zg + u;
                if (z < z1) {
                    const int ic = z * plane + rowc + x;
                    const T pzp = cur.pz[u];
                    T q[4] = {cur.q[u][0], cur.q[u][1], cur.q[u][2], cur.q[u][3]};
                    const T beta = beta_of<T>(cur.m[u]);
                    q[0] = beta * (q[0] - i2h[0] * (cur.pxp[u] - cur.pxm[u]));
                    q[1] = beta * (q[1] - i2h[1] * (cur.pyp[u] - cur.pym[u]));
                    q[2] = beta * (q[2] - i2h[2] * (pzp - pzm));
                    st4(out, ic, q);
                    if (DYN) smax = fmax(smax, sigma_cell(q[0], q[1], q[2], k.ih));
                    pzm = pz0;
                    pz0 = pzp;
                }
            }
            cur = nxt;
        }
    }
    if (DYN && sigma_out) sigma_flush((double)smax, sigma_out);
}

// ------------------------------------------------------------------------------------------------------------
// Reductions (Sec. 3.3).  Each thread accumulates the cells it visits: compensated (TwoSum) sums for the scalar
// inventories, plain per-thread sums of at most 64 terms for energy and squared divergence, an exact room-cell
// count, and the histogram as runs of equal bins (shared atomics only when a run ends).  The CTA epilogue
// combines the warps and writes one partial per quantity; the last CTA to finish (atomic ticket) adds the partials
// in CTA order, so the result does not depend on scheduling.  A NaN or Inf in a field propagates into the energy
// or the scalar total, which the last CTA checks.
//
// Partial sums are float-float pairs on an FP32 grid and doubles on an FP64 grid (Part): GB300 runs FP64 at 1/64
// of the FP32 rate, so the FP32 path stays in float-float arithmetic (about 2^-44 of the sum, exact for counts)
// up to the final values, which the last CTA converts to double once.
//
// With the filter on, the work is split in two launches: the filter records the divergence of its input (the
// projected velocity) per warp (sum of d^2, max |d|), and k_reduce_state reads the filtered state once, flat and
// coalesced, for everything else, folding the filter's divergence records in a fixed order.
// ------------------------------------------------------------------------------------------------------------
template <typename T>
struct Part {
    T s, e;   // running sum and its compensation (a maximum sits in s with e = 0)
    __device__ static Part of(T v) { return {v, T(0)}; }
    __device__ void add(T v)   // one term, TwoSum
    {
        const T t = s + v;
        const T bp = t - s;
        e += (s - (t - bp)) + (v - bp);
        s = t;
    }
    __device__ Part plus(Part b) const   // float-float sum of two pairs
    {
        const T t = s + b.s;
        const T bp = t - s;
        return {t, (e + b.e) + ((s - (t - bp)) + (b.s - bp))};
    }
    __device__ Part maxw(Part b) const { return {fmax(s, b.s), T(0)}; }
    __device__ double value() const { return (double)s + (double)e; }
};

template <>
struct Part<double> {
    double s;
    __device__ static Part of(double v) { return {v}; }
    __device__ void add(double v) { s += v; }
    __device__ Part plus(Part b) const { return {s + b.s}; }
    __device__ Part maxw(Part b) const { return {fmax(s, b.s)}; }
    __device__ double value() const { return s; }
};
static_assert(sizeof(Part<float>) == 8 && sizeof(Part<double>) == 8, "a partial fills one 8-byte slot");

__device__ __forceinline__ Part<float> shfl_part(Part<float> p, int o)
{
    return {__shfl_xor_sync(0xffffffffu, p.s, o), __shfl_xor_sync(0xffffffffu, p.e, o)};
}
__device__ __forceinline__ Part<double> shfl_part(Part<double> p, int o)
{
    return {__shfl_xor_sync(0xffffffffu, p.s, o)};
}
__device__ __forceinline__ Part<float> ld_part(const Part<float>* p)
{
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ Part<double> ld_part(const Part<double>* p)
{
    return {__ldcg(reinterpret_cast<const double*>(p))};
}

// warp-wide sum (fixed butterfly), every lane ends with the total
template <typename T>
__device__ __forceinline__ Part<T> warp_sum(Part<T> p)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) p = p.plus(shfl_part(p, o));
    return p;
}

template <typename T>
__device__ __forceinline__ T warp_maxT(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// histogram bin of a room cell's scalar: kHistBins equal bins on [0, 1], then the counts below 0 and above 1
template <typename T>
__device__ __forceinline__ int hist_bin(T cc)
{
    return cc < T(0) ? kHistBins : (cc > T(1) ? kHistBins + 1 : min((int)(cc * T(kHistBins)), kHistBins - 1));
}

// One thread's counts of its two most recent histogram bins: a shared atomic only when a third bin displaces the
// older one, so a scalar that alternates between two neighbouring bins (noise at a bin edge, or around 1 between
// the top bin and the overflow count) costs no atomics, and the lanes of a warp, which usually share their bins,
// do not serialise on the same counters cell after cell.
struct HistRun {
    int bin0, len0;   // most recent bin
    int bin1, len1;
    __device__ void init() { bin0 = bin1 = -1; len0 = len1 = 0; }
    __device__ __forceinline__ void add(int b, int* hist)
    {
        if (b == bin0) {
            ++len0;
        } else if (b == bin1) {
            const int l = len1 + 1;
            bin1 = bin0; len1 = len0;
            bin0 = b; len0 = l;
        } else {
            if (len1) atomicAdd(&hist[bin1], len1);
            bin1 = bin0; len1 = len0;
            bin0 = b; len0 = 1;
        }
    }
    __device__ void flush(int* hist)
    {
        if (len0) atomicAdd(&hist[bin0], len0);
        if (len1) atomicAdd(&hist[bin1], len1);
    }
};

// Statistics of cells with their divergence (the standalone reductions, filter off)
template <typename T>
struct CellStats {
    Part<T> ct, cr, c2;
    T ke, d2, dmax, umax;
    int vr;
    HistRun run;
    __device__ void init()
    {
        ct = cr = c2 = Part<T>::of(T(0));
        ke = d2 = dmax = umax = T(0);
        vr = 0;
        run.init();
    }
    // q: the cell's (u, v, w, c); d: its divergence; m: its mask byte
    __device__ __forceinline__ void add(const T q[4], T d, uint8_t m, int* hist)
    {
        ke += q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
        d2 += d * d;
        ct.add(q[3]);
        dmax = fmax(dmax, fabs(d));
        umax = fmax(umax, fmax(fabs(q[0]), fmax(fabs(q[1]), fabs(q[2]))));
        if (m & kBitRoom) {
            const T cc = q[3];
            cr.add(cc);
            c2.add(cc * cc);
            ++vr;
            run.add(hist_bin(cc), hist);
        }
    }
};

// Statistics of cells without their divergence (k_reduce_state): the scalar is summed over the room cells and the
// other cells separately (one compensated sum per cell); the total is their sum.
template <typename T>
struct StateStats {
    Part<T> cr, cn, c2;
    T ke, umax;
    int vr;
    HistRun run;
    __device__ void init()
    {
        cr = cn = c2 = Part<T>::of(T(0));
        ke = umax = T(0);
        vr = 0;
        run.init();
    }
    __device__ __forceinline__ void add(const T q[4], uint8_t m, int* hist)
    {
        ke += q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
        umax = fmax(umax, fmax(fabs(q[0]), fmax(fabs(q[1]), fabs(q[2]))));
        const T cc = q[3];
        if (m & kBitRoom) {
            cr.add(cc);
            c2.add(cc * cc);
            ++vr;
            run.add(hist_bin(cc), hist);
        } else {
            cn.add(cc);
        }
    }
};

template <typename T>
struct RedShared {
    int hist[kHistBins + 2];
    long long hist_total[kHistBins + 2];
    Part<T> red[kRedSlots][TX * TY / 32];   // [quantity][warp]
    double fin[kRedSlots];                  // final values (last CTA)
    long long slot;                         // history slot of the record
    bool is_last;
};

template <typename T>
__device__ __forceinline__ void red_init(RedShared<T>& sh)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int i = tid; i < kHistBins + 2; i += TX * TY) sh.hist[i] = 0;
}

// CTA epilogue after the warps have stored their values in sh.red[quantity][warp] and their histogram runs: the
// CTA partials (quantity-major, partial[q * nblocks + cta]), the histogram counters, the ticket, and in the last
// CTA the final sums and the record.  Quantities 0-5 are sums, 6-7 maxima.  SPLIT_C: slot 2 holds the scalar over
// the non-room cells (total = slot 2 + slot 3).  Every thread of a CTA of TX * TY threads calls it once.
// quantities 6 and 7 of the reduction slots are maxima, the others sums
__device__ __forceinline__ bool red_is_max(int q) { return q == 6 || q == 7; }

template <typename T, bool SPLIT_C>
__device__ void red_tail(RedShared<T>& sh, const ReduceArgsDev& r, int to_history)
{
    constexpr int NW = TX * TY / 32;
    static_assert(NW <= kRedSlots && kRedSlots <= 2 * NW, "one or two reduced quantities per warp in the final pass");
    static_assert(TX * TY >= kHistBins + 2, "one thread per histogram counter in the final pass");
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    Part<T>* part = reinterpret_cast<Part<T>*>(r.partial);
    __syncthreads();
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const long long bid = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    if (tid < kRedSlots) {
        Part<T> v = sh.red[tid][0];
        for (int i = 1; i < NW; ++i) v = red_is_max(tid) ? v.maxw(sh.red[tid][i]) : v.plus(sh.red[tid][i]);
        part[(long long)tid * nblocks + bid] = v;
    }
    for (int i = tid; i < kHistBins + 2; i += TX * TY)
        if (sh.hist[i]) atomicAdd(r.hist_accum + i, (unsigned long long)sh.hist[i]);
    __threadfence();
    __syncthreads();
    if (tid == 0) sh.is_last = atomicAdd(r.done, 1u) == (unsigned)(nblocks - 1);
    __syncthreads();
    if (!sh.is_last) return;
    __threadfence();
    // last CTA: every load of the final pass is issued before the first sum.  Warp qq adds partial qq of every CTA
    // in CTA order (lane l: CTAs l, l + 32, ...; then a fixed tree); the histogram counters are read and cleared.
    long long step = 0, count = 0;
    double t_end = 0.0, dt_dyn = 0.0;
    if (tid == 0) {
        step = *r.step_counter;
        if (to_history) count = *r.hist_count;
        if (r.dyn) { t_end = r.dyn->t_end; dt_dyn = r.dyn->dt; }
    }
    if (tid < kHistBins + 2) sh.hist_total[tid] = (long long)atomicExch(r.hist_accum + tid, 0ull);
    for (int qq = wid; qq < kRedSlots; qq += NW) {
        constexpr int kInFlight = 16;
        const bool mx = red_is_max(qq);
        const Part<T>* src = part + (long long)qq * nblocks;
        Part<T> v = Part<T>::of(T(0));   // a sum starts from 0, and so does a maximum (of non-negative values)
        for (int c0 = 0; c0 < nblocks; c0 += 32 * kInFlight) {
            Part<T> pv[kInFlight];
#pragma unroll
            for (int u = 0; u < kInFlight; ++u) {
                const int b = c0 + lane + 32 * u;
                pv[u] = b < nblocks ? ld_part(src + b) : Part<T>::of(T(0));
            }
#pragma unroll
            for (int u = 0; u < kInFlight; ++u) v = mx ? v.maxw(pv[u]) : v.plus(pv[u]);
        }
        v = mx ? Part<T>::of(warp_maxT(v.s)) : warp_sum(v);
        if (lane == 0) sh.fin[qq] = v.value();
    }
    __syncthreads();
    const double c_total = SPLIT_C ? sh.fin[2] + sh.fin[3] : sh.fin[2];
    // the record is written field by field by several threads (no per-thread copy of the whole struct)
    if (tid == 0) sh.slot = to_history ? count % r.history_capacity : 0;
    __syncthreads();
    vf_reduce* outs[2] = {r.out, to_history ? r.history + sh.slot : nullptr};
    for (int o = 0; o < 2; ++o) {
        vf_reduce* dst = outs[o];
        if (!dst) continue;
        for (int i = tid; i < kHistBins + 2; i += TX * TY) {
            if (i < kHistBins) dst->hist[i] = sh.hist_total[i];
            else if (i == kHistBins) dst->hist_under = sh.hist_total[i];
            else dst->hist_over = sh.hist_total[i];
        }
        if (tid == 0) {
            dst->step = step;
            dst->t = r.dyn ? t_end : r.t0 + (double)step * r.dt;
            dst->dt = r.dyn ? dt_dyn : r.dt;
            dst->ke = 0.5 * r.dV * sh.fin[0];
            dst->div_l2 = sqrt(r.dV * sh.fin[1]);
            dst->c_total = r.dV * c_total;
            dst->c_room = r.dV * sh.fin[3];
            dst->c2_room = r.dV * sh.fin[4];
            dst->v_room = r.dV * sh.fin[5];
            dst->div_max = sh.fin[6];
            dst->u_max = sh.fin[7];
            // scalar budget of the step: the stage terms of k_budget, the filter's terms from its records
            dst->budget_forcing = r.budget ? r.budget[0] : 0.0;
            dst->budget_forcing_room = r.budget ? r.budget[1] : 0.0;
            dst->budget_outflow = r.budget ? r.budget[2] : 0.0;
            dst->budget_mask_loss = r.filter_budget ? r.dV * sh.fin[8] : 0.0;
            dst->budget_filter_room = r.filter_budget ? r.dV * sh.fin[9] : 0.0;
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (!isfinite(sh.fin[0]) || !isfinite(c_total)) *r.nonfinite = 1;
        if (to_history) *r.hist_count = count + 1;
        *r.done = 0u;
    }
}

// CTA epilogue of the standalone reductions: warp values of CellStats, then the common tail
template <typename T>
__device__ void red_finish(CellStats<T>& cs, RedShared<T>& sh, const ReduceArgsDev& r, int to_history)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    cs.run.flush(sh.hist);
    const Part<T> ke = warp_sum(Part<T>::of(cs.ke)), d2 = warp_sum(Part<T>::of(cs.d2));
    const Part<T> ct = warp_sum(cs.ct), cr = warp_sum(cs.cr), c2 = warp_sum(cs.c2);
    const int vr = __reduce_add_sync(0xffffffffu, cs.vr);
    const T dmax = warp_maxT(cs.dmax), umax = warp_maxT(cs.umax);
    if (lane == 0) {
        sh.red[0][wid] = ke;
        sh.red[1][wid] = d2;
        sh.red[2][wid] = ct;
        sh.red[3][wid] = cr;
        sh.red[4][wid] = c2;
        sh.red[5][wid] = Part<T>::of((T)vr);   // at most 32 x 64 cells: exact
        sh.red[6][wid] = Part<T>::of(dmax);
        sh.red[7][wid] = Part<T>::of(umax);
        sh.red[8][wid] = Part<T>::of(T(0));   // no filter records
        sh.red[9][wid] = Part<T>::of(T(0));
    }
    red_tail<T, false>(sh, r, to_history);
}

// Standalone reductions of a state (filter off, or on demand): divergence of the state itself.
template <typename T>
__global__ void __launch_bounds__(TX * TY) k_reduce(const void* __restrict__ q, const uint8_t* __restrict__ mask,
                                                    FlowConsts<T> k, ReduceArgsDev r, int to_history)
{
    pdl_enter();
    __shared__ RedShared<T> sh;
    red_init(sh);
    __syncthreads();
    CellStats<T> cs;
    cs.init();
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x < k.nx && y < k.ny) {
        const int nx = k.nx, ny = k.ny, nz = k.nz;
        const int plane = nx * ny;
        const int z0 = blockIdx.z * k.zc[kZcFilter], z1 = min(z0 + k.zc[kZcFilter], nz);
        const int rowc = y * nx, rowm = wrap(y - 1, ny) * nx, rowp = wrap(y + 1, ny) * nx;
        const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
        T wzm = ld1<T>(q, wrap(z0 - 1, nz) * plane + rowc + x, 2);
        T c4[4], n4[4];
        ld4(q, z0 * plane + rowc + x, c4);
        ld4(q, wrap(z0 + 1, nz) * plane + rowc + x, n4);
        for (int z = z0; z < z1; ++z) {
            const int zb = z * plane;
            T nn4[4] = {T(0), T(0), T(0), T(0)};
            if (z + 1 < z1) ld4(q, wrap(z + 2, nz) * plane + rowc + x, nn4);   // prefetch
            const T d = k.i2h[0] * (ld1<T>(q, zb + rowc + xp, 0) - ld1<T>(q, zb + rowc + xm, 0)) +
                        k.i2h[1] * (ld1<T>(q, zb + rowp + x, 1) - ld1<T>(q, zb + rowm + x, 1)) +
                        k.i2h[2] * (n4[2] - wzm);
            cs.add(c4, d, __ldg(mask + zb + rowc + x), sh.hist);
            wzm = c4[2];
#pragma unroll
            for (int f = 0; f < 4; ++f) { c4[f] = n4[f]; n4[f] = nn4[f]; }
        }
    }
    red_finish(cs, sh, r, to_history);
}

// Reductions of the filtered state (filter on): each CTA takes one contiguous chunk of cpt * kRedThreads cells
// (cpt <= kRedMaxCellsPerThread cells per thread, consecutive threads on consecutive cells), the grid one full
// wave of CTAs where that bound allows; plus the filter's per-warp divergence records (r.div_count of them, each
// {sum d^2, max |d|}), folded by the threads in a fixed order.
constexpr int kRedMaxCellsPerThread = 64;
constexpr int kRedBatch = 4;
constexpr int kRedThreads = TX * TY;

template <typename T>
__global__ void __launch_bounds__(kRedThreads, sizeof(T) == 4 ? 4 : 2)
k_reduce_state(const void* __restrict__ q, const uint8_t* __restrict__ mask, int n, int cpt, ReduceArgsDev r,
               int to_history)
{
    pdl_enter();
    __shared__ RedShared<T> sh;
    red_init(sh);
    __syncthreads();
    StateStats<T> cs;
    cs.init();
    const int tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const int base = blockIdx.x * (kRedThreads * cpt) + tid;
    // batches of kRedBatch cells, software-pipelined: the loads of the next batch are issued before the current
    // batch is accumulated (its histogram atomics would otherwise hold the loads back); a cell past the chunk or the
    // grid reads as zeros outside the room, which adds nothing
    auto load_batch = [&](int j0, T (&c4)[kRedBatch][4], uint8_t (&m)[kRedBatch]) {
#pragma unroll
        for (int u = 0; u < kRedBatch; ++u) {
            const int i = base + (j0 + u) * kRedThreads;
            if (j0 + u < cpt && i < n) {
                ld4(q, i, c4[u]);
                m[u] = __ldg(mask + i);
            } else {
                c4[u][0] = c4[u][1] = c4[u][2] = c4[u][3] = T(0);
                m[u] = 0;
            }
        }
    };
    T cur[kRedBatch][4], nxt[kRedBatch][4];
    uint8_t mcur[kRedBatch], mnxt[kRedBatch];
    load_batch(0, cur, mcur);
    for (int j0 = 0; j0 < cpt; j0 += kRedBatch) {
        load_batch(j0 + kRedBatch, nxt, mnxt);
#pragma unroll
        for (int u = 0; u < kRedBatch; ++u) cs.add(cur[u], mcur[u], sh.hist);
#pragma unroll
        for (int u = 0; u < kRedBatch; ++u) {
            mcur[u] = mnxt[u];
#pragma unroll
            for (int f = 0; f < 4; ++f) cur[u][f] = nxt[u][f];
        }
    }
    // the filter's records (divergence, mask loss, room change), folded in record order per thread
    Part<T> d2 = Part<T>::of(T(0)), ml = Part<T>::of(T(0)), fr = Part<T>::of(T(0));
    T dmax = T(0);
    const Part<T>* rec = reinterpret_cast<const Part<T>*>(r.div_partial);
    for (int j = blockIdx.x * kRedThreads + tid; j < r.div_count; j += gridDim.x * kRedThreads) {
        const Part<T>* rj = rec + kDivRecord * (long long)j;
        d2 = d2.plus(ld_part(rj));
        dmax = fmax(dmax, ld_part(rj + 1).s);
        ml = ml.plus(ld_part(rj + 2));
        fr = fr.plus(ld_part(rj + 3));
    }
    cs.run.flush(sh.hist);
    const Part<T> ke = warp_sum(Part<T>::of(cs.ke));
    const Part<T> cn = warp_sum(cs.cn), cr = warp_sum(cs.cr), c2 = warp_sum(cs.c2);
    d2 = warp_sum(d2);
    ml = warp_sum(ml);
    fr = warp_sum(fr);
    const int vr = __reduce_add_sync(0xffffffffu, cs.vr);
    const T umax = warp_maxT(cs.umax);
    dmax = warp_maxT(dmax);
    if (lane == 0) {
        sh.red[0][wid] = ke;
        sh.red[1][wid] = d2;
        sh.red[2][wid] = cn;
        sh.red[3][wid] = cr;
        sh.red[4][wid] = c2;
        sh.red[5][wid] = Part<T>::of((T)vr);   // at most 32 x 64 cells: exact
        sh.red[6][wid] = Part<T>::of(dmax);
        sh.red[7][wid] = Part<T>::of(umax);
        sh.red[8][wid] = ml;
        sh.red[9][wid] = fr;
    }
    red_tail<T, true>(sh, r, to_history);
}

// ------------------------------------------------------------------------------------------------------------
// Sixth-order filter q <- beta (q + pi^-6 sum_j S6_j q), S6 = (1, -6, 15, -20, 15, -6, 1) (Eq. 6).
// DIVSTAT: also the divergence of the filter's input (the projected velocity, after the projection and before the
// filter) for the reductions (Sec. 3.3), and the filter's share of the scalar budget: per warp the sum of d^2,
// max |d|, the sum over solid cells of the unmasked filtered scalar (what the re-mask removes) and the sum over
// fluid room cells of the filter's change of the scalar, into r.div_partial (kDivRecord values), no CTA barrier.
// ------------------------------------------------------------------------------------------------------------
template <typename T, bool DIVSTAT, bool SIGMA>
__global__ void __launch_bounds__(TX * filter_ty<T>(), sizeof(T) == 4 ? 32 / filter_ty<T>() : 2)
k_filter(const void* __restrict__ in, void* __restrict__ out, const uint8_t* __restrict__ mask, FlowConsts<T> k,
         ReduceArgsDev r, unsigned long long* sigma_out)
{
    pdl_enter();
    // x / y neighbours from a shared-memory tile of the current plane: the CTA's TX x FY cells and a 3-cell halo
    // ring (periodic), double buffered; the ring of the next plane arrives by cp.async while the current plane is
    // filtered, the interior is each thread's own z-window register.  The z neighbours stay in registers.
    // Three buffers in FP32 (a buffer is refilled two planes after it was read, so one CTA barrier per plane
    // suffices); two in FP64 (within the static shared-memory limit: a second barrier guards the refill).
    constexpr int FY = filter_ty<T>();
    constexpr int HW = TX + 6, HH = FY + 6, V = 4 * (int)sizeof(T) / 16;   // 16-byte pieces per 4-vector
    constexpr int NB = sizeof(T) == 4 ? 3 : 2;
    __shared__ __align__(16) T tile[NB][HH][HW][4];
    T smax = T(0);   // SIGMA: Courant rate of the filtered velocity (the step's final state)
    T d2 = T(0), dmax = T(0), mloss = T(0), froom = T(0);
    const int nx = k.nx, ny = k.ny, nz = k.nz;
    const int plane = nx * ny;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * FY;
    const int x = x0 + tx, y = y0 + ty;
    const bool act = x < nx && y < ny;
    const int wx = min(TX, nx - x0), wy = min(FY, ny - y0);   // cells of this (possibly ragged) tile
    const int W = wx + 6, H = wy + 6;
    const int z0 = blockIdx.z * k.zc[kZcFilter], z1 = min(z0 + k.zc[kZcFilter], nz);
    // The halo ring: tile cell (sx, sy) holds cell (x0 + sx - 3, y0 + sy - 3), wrapped.  The ring has at most
    // 2 (TX + FY + 6) * 3 <= 2 TX FY cells; thread tid owns ring cells tid and tid + TX FY (in ring order), whose
    // in-plane cell index and shared-memory offset are found once.
    constexpr int kRingMax = 2;
    int ring_cell[kRingMax];
    uint32_t ring_smem[kRingMax];
    {
        const int n_ring = W * H - wx * wy;
        for (int o = 0; o < kRingMax; ++o) {
            const int j = tid + o * TX * FY;
            ring_cell[o] = -1;
            ring_smem[o] = 0u;
            if (j >= n_ring) continue;
            // ring order: the 3 rows above, then 3 + 3 cells on each interior row, then the 3 rows below
            int sx, sy;
            if (j < 3 * W) { sy = j / W; sx = j - sy * W; }
            else if (j < 3 * W + 6 * wy) { const int q = j - 3 * W; sy = 3 + q / 6; const int c = q - (q / 6) * 6; sx = c < 3 ? c : wx + c; }
            else { const int q = j - 3 * W - 6 * wy; sy = wy + 3 + q / W; sx = q - (q / W) * W; }
            ring_cell[o] = wrap(y0 + sy - 3, ny) * nx + wrap(x0 + sx - 3, nx);
            ring_smem[o] = (uint32_t)__cvta_generic_to_shared(&tile[0][sy][sx][0]);
        }
    }
    constexpr uint32_t kTileBytes = (uint32_t)sizeof(tile[0]);
    auto ring = [&](int zz, int b) {
        const size_t zb = (size_t)zz * plane;
#pragma unroll
        for (int o = 0; o < kRingMax; ++o) {
            if (ring_cell[o] < 0) continue;
            const char* src = reinterpret_cast<const char*>(in) + (zb + ring_cell[o]) * 4 * sizeof(T);
            const uint32_t dst = ring_smem[o] + (uint32_t)b * kTileBytes;
#pragma unroll
            for (int v = 0; v < V; ++v)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16u * v), "l"(src + 16 * v)
                             : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const int yc = (act ? y : 0) * nx, xa = act ? x : 0;
    // z window of 7 planes of the 4-vector, in registers
    T zw[7][4] = {};
    if (act) {
#pragma unroll
        for (int m = 0; m < 6; ++m) ld4(in, wrap(z0 + m - 3, nz) * plane + yc + xa, zw[m + 1]);
    }
    if (z0 < z1) ring(z0, 0);
    int s = 0;
    for (int z = z0; z < z1; ++z) {
        const int zb = z * plane;
        const int ic = zb + yc + xa;
#pragma unroll
        for (int m = 0; m < 6; ++m)
#pragma unroll
            for (int f = 0; f < 4; ++f) zw[m][f] = zw[m + 1][f];
        if (act) ld4(in, wrap(z + 3, nz) * plane + yc + xa, zw[6]);
        if (NB == 2) __syncthreads();           // every read of the other buffer (plane z - 1) is done
        const int sn = s + 1 == NB ? 0 : s + 1;
        if (z + 1 < z1) ring(z + 1, sn);
        else asm volatile("cp.async.commit_group;" ::: "memory");   // an empty group keeps the wait count uniform
        if (act) {
#pragma unroll
            for (int f = 0; f < 4; ++f) tile[s][ty + 3][tx + 3][f] = zw[3][f];
        }
        asm volatile("cp.async.wait_group 1;" ::: "memory");   // this thread's ring copies of plane z
        __syncthreads();
        if (act) {
            // sum of the three sixth differences: sum_m S6[m] (q_x[m] + q_y[m] + q_z[m]); centre weight -20 x 3
            T acc[4];
#pragma unroll
            for (int f = 0; f < 4; ++f)
                acc[f] = (zw[0][f] + zw[6][f]) - T(6) * (zw[1][f] + zw[5][f]) + T(15) * (zw[2][f] + zw[4][f]) -
                         T(60) * zw[3][f];
            const T coef[3] = {T(1), T(-6), T(15)};
            T div = T(0);
#pragma unroll
            for (int d = 3; d >= 1; --d) {
                const T cf = coef[3 - d];
                T a[4], b[4], c[4], e[4];
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    a[f] = tile[s][ty + 3][tx + 3 - d][f];
                    b[f] = tile[s][ty + 3][tx + 3 + d][f];
                    c[f] = tile[s][ty + 3 - d][tx + 3][f];
                    e[f] = tile[s][ty + 3 + d][tx + 3][f];
                }
#pragma unroll
                for (int f = 0; f < 4; ++f) acc[f] += cf * ((a[f] + b[f]) + (c[f] + e[f]));
                if (DIVSTAT && d == 1)
                    div = k.i2h[0] * (b[0] - a[0]) + k.i2h[1] * (e[1] - c[1]) + k.i2h[2] * (zw[4][2] - zw[2][2]);
            }
            const uint8_t m0 = __ldg(mask + ic);
            const T beta = beta_of<T>(m0);
            T o[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) o[f] = beta * (zw[3][f] + k.filt * acc[f]);
            st4(out, ic, o);
            if (DIVSTAT) {
                d2 += div * div;
                dmax = fmax(dmax, fabs(div));
                const T change = k.filt * acc[3];
                if (!(m0 & kBitBeta)) mloss += zw[3][3] + change;
                else if (m0 & kBitRoom) froom += change;
            }
            if (SIGMA) smax = fmax(smax, sigma_cell(o[0], o[1], o[2], k.ih));
        }
        s = sn;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (SIGMA) sigma_flush((double)smax, sigma_out);
    if (DIVSTAT) {
        const Part<T> s = warp_sum(Part<T>::of(d2));
        const T m = warp_maxT(dmax);
        const Part<T> ml = warp_sum(Part<T>::of(mloss)), fr = warp_sum(Part<T>::of(froom));
        if ((tid & 31) == 0) {
            const long long bid = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
            const long long w = bid * (TX * FY / 32) + (tid >> 5);
            Part<T>* rec = reinterpret_cast<Part<T>*>(r.div_partial) + kDivRecord * w;
            rec[0] = s;
            rec[1] = Part<T>::of(m);
            rec[2] = ml;
            rec[3] = fr;
        }
    }
}

// ------------------------------------------------------------------------------------------------------------
// Smooth source mask (Eq. 5): S = prod_j (1 - tanh(B_j [d_j / (W_j/2) - (W_j/2) / d_j])) / 2, d_j the
// minimum-image distance from the cell centre i h_j to c_j; the factor is its limit 1 where d_j = 0.  Evaluated
// in double, stored in the grid's precision; the mask's S bit marks S > 0.
// ------------------------------------------------------------------------------------------------------------
__device__ __forceinline__ double tanh_factor(int i, int j, const TanhWindow& w)
{
    double d = fabs((double)i * w.h[j] - w.c[j]);
    d = fmin(d, w.L[j] - d);
    if (!(d > 0.0)) return 1.0;
    return 0.5 * (1.0 - tanh(w.B[j] * (d / w.hw[j] - w.hw[j] / d)));
}

template <typename T>
__global__ void k_tanh_source(T* __restrict__ sval, uint8_t* __restrict__ mask, TanhWindow w, int nx, int ny, int nz)
{
    const size_t n = (size_t)nx * ny * nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        const double S = ((1.0 * tanh_factor(x, 0, w)) * tanh_factor(y, 1, w)) * tanh_factor(z, 2, w);
        const T v = (T)S;
        sval[i] = v;
        mask[i] = (uint8_t)((mask[i] & ~kBitS) | (v > T(0) ? kBitS : 0));
    }
}

template <typename T>
__global__ void k_source_bits(uint8_t* __restrict__ mask, const T* __restrict__ sval, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        mask[i] = (uint8_t)((mask[i] & ~kBitS) | (sval[i] > T(0) ? kBitS : 0));
}

// ------------------------------------------------------------------------------------------------------------
// Immersed-boundary force on a region: F_i = dV sum_region [-conv_i + nu diff_i + S (target_i - u_i) / tau_f + b_i
// - delta_i p], the unmasked right-hand side of Eq. 2 in FP64 (the rate at which the mask removes momentum there)
// ------------------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_region_force(const void* __restrict__ q, const T* __restrict__ p,
                                                      const uint8_t* __restrict__ mask, const T* __restrict__ sval,
                                                      const void* __restrict__ target, FlowConsts<T> k, double dV,
                                                      double* acc)
{
    const size_t n = (size_t)k.nx * k.ny * k.nz;
    const double inv_tau = k.dyn ? k.dyn->inv_tau : (double)k.inv_tau;
    double F[3] = {0.0, 0.0, 0.0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint8_t m = mask[i];
        if (!(m & kBitForce)) continue;
        const int x = (int)(i % k.nx), y = (int)((i / k.nx) % k.ny), z = (int)(i / ((size_t)k.nx * k.ny));
        const int plane = k.nx * k.ny;
        const int im[3] = {z * plane + y * k.nx + wrap(x - 1, k.nx), z * plane + wrap(y - 1, k.ny) * k.nx + x,
                           wrap(z - 1, k.nz) * plane + y * k.nx + x};
        const int ip[3] = {z * plane + y * k.nx + wrap(x + 1, k.nx), z * plane + wrap(y + 1, k.ny) * k.nx + x,
                           wrap(z + 1, k.nz) * plane + y * k.nx + x};
        T tc[4], tm[3][4], tp[3][4];
        ld4(q, (int)i, tc);
        for (int j = 0; j < 3; ++j) { ld4(q, im[j], tm[j]); ld4(q, ip[j], tp[j]); }
        double c[3], qm[3][3], qp[3][3];
        for (int a = 0; a < 3; ++a) {
            c[a] = tc[a];
            for (int j = 0; j < 3; ++j) { qm[j][a] = tm[j][a]; qp[j][a] = tp[j][a]; }
        }
        double S = 0.0, tgt[3] = {(double)k.uset[0], (double)k.uset[1], (double)k.uset[2]};
        if (m & kBitS) {
            S = sval ? (double)sval[i] : 1.0;
            if (target) {
                T t4[4];
                ld4(target, (int)i, t4);
                for (int a = 0; a < 3; ++a) tgt[a] = t4[a];
            }
        }
        for (int a = 0; a < 3; ++a) {
            double conv = 0.0, diff = 0.0;
            for (int j = 0; j < 3; ++j) {
                const double i2h = (double)k.i2h[j];
                conv += 0.5 * ((qp[j][j] * qp[j][a] - qm[j][j] * qm[j][a]) * i2h + c[j] * (qp[j][a] - qm[j][a]) * i2h);
                diff += (qp[j][a] - 2.0 * c[a] + qm[j][a]) * (double)k.ih2[j];
            }
            const double grad_p = ((double)p[ip[a]] - (double)p[im[a]]) * (double)k.i2h[a];
            const double rhs = -conv + (double)k.nu * diff + S * (tgt[a] - c[a]) * inv_tau + (double)k.bf[a] - grad_p;
            F[a] += rhs * dV;
        }
    }
    __shared__ double part[3][8];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int a = 0; a < 3; ++a) {
        double v = F[a];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) part[a][wid] = v;
    }
    __syncthreads();
    if (tid < 3) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += part[tid][w];
        if (v != 0.0) atomicAdd(acc + tid, v);
    }
}

// ------------------------------------------------------------------------------------------------------------
// Dynamic time step (Sec. 2.4): the Courant rate of a state, and the adjust kernel at the start of a step
// ------------------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_courant_rate(const void* __restrict__ q, FlowConsts<T> k, size_t n,
                                                      unsigned long long* sigma)
{
    pdl_enter();
    T smax = T(0);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        T v[4];
        ld4(q, (int)i, v);
        smax = fmax(smax, sigma_cell(v[0], v[1], v[2], k.ih));
    }
    sigma_flush((double)smax, sigma);
}

// dt = min(dt_max, courant_max / sigma) (dt_max at rest), then the dt-dependent constants with the formulas the
// host uses for a fixed dt, the time at the end of the step, and a cleared sigma for the step's last kernel
__global__ void k_adjust_dt(DtCtl* c)
{
    pdl_enter();
    // lane 0 chooses dt; the lanes then form one dt-dependent constant each (the divisions run side by side)
    const int lane = threadIdx.x;
    double dt = 0.0;
    if (lane == 0) {
        const double sigma = __longlong_as_double((long long)c->sigma_bits);
        dt = c->dt_max;
        if (sigma > 0.0) {
            const double lim = c->courant_max / sigma;
            if (lim < dt) dt = lim;
        }
    }
    dt = __shfl_sync(0xffffffffu, dt, 0);
    switch (lane) {
        case 0: c->dt = dt; c->t_end = c->t_end + dt; c->sigma_bits = 0ull; break;
        case 1: c->dt2 = dt / 2.0; break;
        case 2: c->dt3 = dt / 3.0; break;
        case 3: c->dt6 = dt / 6.0; break;
        case 4: c->inv_tau = 1.0 / (c->tau_f > 0.0 ? c->tau_f : dt); break;
        case 5: case 6: case 7: c->i2h_div[lane - 5] = 1.0 / (2.0 * c->h[lane - 5] * dt); break;
        case 8: case 9: case 10: c->i2h_dt[lane - 8] = dt / (2.0 * c->h[lane - 8]); break;
        default: break;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Conversions and masks
// ------------------------------------------------------------------------------------------------------------
// dst[i] (component comp of a 4-vector array, or a scalar array when comp < 0) = src[i] * scale, zero in solids
// when a mask is given
template <typename Tin, typename Tout>
__global__ void k_convert_in(const Tin* __restrict__ src, Tout* __restrict__ dst, int comp, size_t n, double scale,
                             const uint8_t* __restrict__ mask)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double v = (double)src[i] * scale;
        if (mask && !(mask[i] & kBitBeta)) v = 0.0;
        dst[comp < 0 ? i : 4 * i + comp] = (Tout)v;
    }
}

template <typename Tin, typename Tout>
__global__ void k_convert_out(const Tin* __restrict__ src, int comp, Tout* __restrict__ dst, size_t n, double scale)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (Tout)((double)src[comp < 0 ? i : 4 * i + comp] * scale);
}

template <typename T>
__global__ void k_apply_mask4(T* q, const uint8_t* __restrict__ mask, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(mask[i] & kBitBeta))
#pragma unroll
            for (int f = 0; f < 4; ++f) q[4 * i + f] = T(0);
}

__global__ void k_mask_merge(uint8_t* mask, const uint8_t* __restrict__ src, uint8_t bit, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        mask[i] = (uint8_t)((mask[i] & ~bit) | (src[i] ? bit : 0));
}

__global__ void k_mask_fill(uint8_t* mask, uint8_t value, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        mask[i] = value;
}

__global__ void k_count_solid(const uint8_t* __restrict__ mask, size_t n, unsigned long long* count)
{
    unsigned long long local = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        local += (mask[i] & kBitBeta) ? 0 : 1;
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

// stencil mask: own beta and S, and the beta of the six axis neighbours
__global__ void k_build_smask(const uint8_t* __restrict__ mask, uint8_t* __restrict__ smask, int nx, int ny, int nz)
{
    const size_t n = (size_t)nx * ny * nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        const size_t plane = (size_t)nx * ny, row = (size_t)y * nx, zb = (size_t)z * plane;
        const uint8_t m = mask[i];
        auto fl = [&](size_t j, uint8_t bit) { return (mask[j] & kBitBeta) ? bit : (uint8_t)0; };
        uint8_t b = (uint8_t)(((m & kBitBeta) ? kSmSelf : 0) | ((m & kBitS) ? kSmS : 0));
        b |= fl(zb + row + wrap(x - 1, nx), kSmXm) | fl(zb + row + wrap(x + 1, nx), kSmXp);
        b |= fl(zb + (size_t)wrap(y - 1, ny) * nx + x, kSmYm) | fl(zb + (size_t)wrap(y + 1, ny) * nx + x, kSmYp);
        b |= fl((size_t)wrap(z - 1, nz) * plane + row + x, kSmZm) | fl((size_t)wrap(z + 1, nz) * plane + row + x, kSmZp);
        smask[i] = b;
    }
}

// bit 3 of every cell: set when one of its six axis neighbours is solid (beta = 0)
__global__ void k_mark_near_solid(uint8_t* mask, int nx, int ny, int nz)
{
    const size_t n = (size_t)nx * ny * nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        const size_t plane = (size_t)nx * ny, row = (size_t)y * nx, zb = (size_t)z * plane;
        const bool solid_nb =
            !(mask[zb + row + wrap(x - 1, nx)] & kBitBeta) || !(mask[zb + row + wrap(x + 1, nx)] & kBitBeta) ||
            !(mask[zb + (size_t)wrap(y - 1, ny) * nx + x] & kBitBeta) ||
            !(mask[zb + (size_t)wrap(y + 1, ny) * nx + x] & kBitBeta) ||
            !(mask[(size_t)wrap(z - 1, nz) * plane + row + x] & kBitBeta) ||
            !(mask[(size_t)wrap(z + 1, nz) * plane + row + x] & kBitBeta);
        mask[i] = (uint8_t)((mask[i] & ~kBitNearSolid) | (solid_nb ? kBitNearSolid : 0));
    }
}

// budget bit of every cell: a fluid forcing cell, or a fluid room cell with a fluid axis neighbour outside the room
__global__ void k_mark_budget(uint8_t* mask, int nx, int ny, int nz)
{
    const size_t n = (size_t)nx * ny * nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
        const size_t plane = (size_t)nx * ny, row = (size_t)y * nx, zb = (size_t)z * plane;
        const uint8_t m = mask[i];
        bool flag = false;
        if (m & kBitBeta) {
            flag = (m & kBitS) != 0;
            if (!flag && (m & kBitRoom)) {
                auto open = [&](size_t j) { return (mask[j] & (kBitBeta | kBitRoom)) == kBitBeta; };
                flag = open(zb + row + wrap(x - 1, nx)) || open(zb + row + wrap(x + 1, nx)) ||
                       open(zb + (size_t)wrap(y - 1, ny) * nx + x) || open(zb + (size_t)wrap(y + 1, ny) * nx + x) ||
                       open((size_t)wrap(z - 1, nz) * plane + row + x) || open((size_t)wrap(z + 1, nz) * plane + row + x);
            }
        }
        mask[i] = (uint8_t)((m & ~kBitBudget) | (flag ? kBitBudget : 0));
    }
}

__global__ void k_list_counts(const uint8_t* __restrict__ mask, size_t n, uint8_t bit, int* counts)
{
    __shared__ int warp_tot[kListChunk / 32];
    const size_t base = (size_t)blockIdx.x * kListChunk;
    int local = 0;
    for (int t = threadIdx.x; t < kListChunk; t += blockDim.x) {
        const size_t i = base + t;
        if (i < n && (mask[i] & bit)) ++local;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += warp_tot[w];
        counts[blockIdx.x] = s;
    }
}

// each chunk writes its flagged cells in ascending order from its offset (ballot + popcount prefix per warp)
__global__ void k_list_fill(const uint8_t* __restrict__ mask, size_t n, uint8_t bit, const int* __restrict__ offsets,
                            int* list)
{
    __shared__ int warp_tot[32];
    __shared__ int running;
    const size_t base = (size_t)blockIdx.x * kListChunk;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) running = offsets[blockIdx.x];
    __syncthreads();
    for (int r = 0; r < kListChunk; r += blockDim.x) {
        const size_t i = base + r + threadIdx.x;
        const bool flag = i < n && (mask[i] & bit);
        const unsigned bal = __ballot_sync(0xffffffffu, flag);
        if (lane == 0) warp_tot[wid] = __popc(bal);
        __syncthreads();
        int before = running;
        for (int w = 0; w < wid; ++w) before += warp_tot[w];
        if (flag) list[before + __popc(bal & ((1u << lane) - 1u))] = (int)i;
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int w = 0; w < nw; ++w) s += warp_tot[w];
            running += s;
        }
        __syncthreads();
    }
}

template <typename T>
inline dim3 flow_grid(const FlowConsts<T>& k, int kind, int ty = TY)
{
    const int zc = k.zc[kind];
    return dim3((k.nx + TX - 1) / TX, (k.ny + ty - 1) / ty, (k.nz + zc - 1) / zc);
}

inline int elementwise_blocks(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

}  // namespace

bool pdl_on()
{
    static const bool on = [] {
        const char* v = std::getenv("VF_PDL");
        return v && *v && *v != '0';
    }();
    return on;
}

// ------------------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------------------
template <typename T>
int Kernels<T>::budget_cta_capacity(const FlowConsts<T>& k)
{
    const dim3 g = flow_grid(k, kZcStage);
    return (int)(g.x * g.y);
}

template <typename T>
cudaError_t Kernels<T>::stage(int s, const StageArgs<T>& a, const FlowConsts<T>& k, cudaStream_t st)
{
    dim3 g = flow_grid(k, kZcStage);
    const dim3 b(TX, TY);
    if (s >= 3 && a.bud.n >= 0) {
        if (a.bud.ctas < 1 || a.bud.ctas > (int)(g.x * g.y) || a.bud.ctas > a.bud.cap) return cudaErrorInvalidValue;
        g.z += 1;   // the budget slice
    }
    const bool dyn = k.dyn != nullptr;
    switch (s) {
        case 1: return launch_pdl(dyn ? k_stage<T, 1, true> : k_stage<T, 1, false>, g, b, 0, st, a, k);
        case 2: return launch_pdl(dyn ? k_stage<T, 2, true> : k_stage<T, 2, false>, g, b, 0, st, a, k);
        case 3: return launch_pdl(dyn ? k_stage<T, 3, true> : k_stage<T, 3, false>, g, b, 0, st, a, k);
        case 4: return launch_pdl(dyn ? k_stage<T, 4, true> : k_stage<T, 4, false>, g, b, 0, st, a, k);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t Kernels<T>::divergence(const void* qstar, T* r, const FlowConsts<T>& k, cudaStream_t st)
{
    return launch_pdl(k.dyn ? k_div<T, true> : k_div<T, false>, flow_grid(k, kZcDiv), dim3(TX, TY), 0, st, qstar, r,
                      k);
}

template <typename T>
cudaError_t Kernels<T>::project(const void* qstar, const T* p, void* out, const uint8_t* mask,
                                long long* step_counter, const FlowConsts<T>& k, cudaStream_t st,
                                unsigned long long* sigma)
{
    const dim3 g = flow_grid(k, kZcProject), b(TX, TY);
    if (k.dyn) return launch_pdl(k_project<T, true>, g, b, 0, st, qstar, p, out, mask, step_counter, k, sigma);
    return launch_pdl(k_project<T, false>, g, b, 0, st, qstar, p, out, mask, step_counter, k,
                      (unsigned long long*)nullptr);
}

template <typename T>
cudaError_t Kernels<T>::filter(const void* in, void* out, const uint8_t* mask, const FlowConsts<T>& k,
                               const ReduceArgsDev* r, cudaStream_t st, unsigned long long* sigma)
{
    const dim3 g = flow_grid(k, kZcFilter, filter_ty<T>()), b(TX, filter_ty<T>());
    const ReduceArgsDev ra = r ? *r : ReduceArgsDev{};
    auto kern = r ? (sigma ? k_filter<T, true, true> : k_filter<T, true, false>)
                  : (sigma ? k_filter<T, false, true> : k_filter<T, false, false>);
    return launch_pdl(kern, g, b, 0, st, in, out, mask, k, ra, sigma);
}

template <typename T>
int Kernels<T>::filter_warps(const FlowConsts<T>& k)
{
    const dim3 g = flow_grid(k, kZcFilter, filter_ty<T>());
    return (int)(g.x * g.y * g.z) * (TX * filter_ty<T>() / 32);
}

template <typename T>
cudaError_t Kernels<T>::reduce_state(const void* q, const uint8_t* mask, const FlowConsts<T>& k, ReduceArgsDev r,
                                     int to_history, int max_blocks, cudaStream_t st)
{
    // one full wave: SMs x resident CTAs (queried once per device), more waves only where a wave would give a
    // thread more than kRedMaxCellsPerThread cells; never more CTAs than partial slots
    static int wave[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!wave[dev]) {
        int sms = 0, per_sm = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_reduce_state<T>, kRedThreads, 0)) !=
            cudaSuccess)
            return e;
        wave[dev] = std::max(1, sms * std::max(1, per_sm));
    }
    const long long n = (long long)k.nx * k.ny * k.nz;
    const long long rows = (n + kRedThreads - 1) / kRedThreads;   // cells per thread if there were one CTA
    long long nb = wave[dev];
    while (nb * kRedMaxCellsPerThread < rows) nb += wave[dev];
    nb = std::min(nb, std::min(rows, (long long)max_blocks));
    const int cpt = (int)((rows + nb - 1) / nb);
    if (cpt > kRedMaxCellsPerThread) return cudaErrorInvalidValue;   // too few partial slots for this grid
    nb = (rows + cpt - 1) / cpt;
    r.div_count = filter_warps(k);
    return launch_pdl(k_reduce_state<T>, dim3((unsigned)nb), dim3(kRedThreads), 0, st, q, mask, (int)n, cpt, r,
                      to_history);
}

template <typename T>
cudaError_t Kernels<T>::tanh_source(T* sval, uint8_t* mask, const TanhWindow& w, int nx, int ny, int nz,
                                    cudaStream_t st)
{
    k_tanh_source<T><<<elementwise_blocks((size_t)nx * ny * nz), 256, 0, st>>>(sval, mask, w, nx, ny, nz);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::source_bits(uint8_t* mask, const T* sval, size_t n, cudaStream_t st)
{
    k_source_bits<T><<<elementwise_blocks(n), 256, 0, st>>>(mask, sval, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::courant_rate(const void* q, const FlowConsts<T>& k, size_t n, unsigned long long* sigma,
                                     cudaStream_t st)
{
    k_courant_rate<T><<<elementwise_blocks(n), 256, 0, st>>>(q, k, n, sigma);
    return cudaGetLastError();
}

template <typename T>
cudaError_t region_force(const void* q, const T* p, const uint8_t* mask, const T* sval, const void* target,
                         const FlowConsts<T>& k, double dV, double* acc, cudaStream_t st)
{
    const size_t n = (size_t)k.nx * k.ny * k.nz;
    k_region_force<T><<<elementwise_blocks(n), 256, 0, st>>>(q, p, mask, sval, target, k, dV, acc);
    return cudaGetLastError();
}
template cudaError_t region_force<float>(const void*, const float*, const uint8_t*, const float*, const void*,
                                         const FlowConsts<float>&, double, double*, cudaStream_t);
template cudaError_t region_force<double>(const void*, const double*, const uint8_t*, const double*, const void*,
                                          const FlowConsts<double>&, double, double*, cudaStream_t);

cudaError_t adjust_dt(DtCtl* c, cudaStream_t st)
{
    return launch_pdl(k_adjust_dt, dim3(1), dim3(32), 0, st, c);   // one warp
}

template <typename T>
int Kernels<T>::reduce_blocks(const FlowConsts<T>& k)
{
    // the most CTAs any allowed filter/reduce z-chunk launches: the smallest chunk (k_reduce_state launches fewer)
    FlowConsts<T> c = k;
    c.zc[kZcFilter] = kZChunkMin;
    const dim3 g = flow_grid(c, kZcFilter);
    return (int)(g.x * g.y * g.z);
}

template <typename T>
cudaError_t Kernels<T>::reduce(const void* q, const uint8_t* mask, const FlowConsts<T>& k, const ReduceArgsDev& r,
                               int to_history, cudaStream_t st)
{
    return launch_pdl(k_reduce<T>, flow_grid(k, kZcFilter), dim3(TX, TY), 0, st, q, mask, k, r, to_history);
}

template <typename T>
cudaError_t Kernels<T>::convert_in(const void* src, int src_fp64, void* dst, int comp, size_t n, double scale,
                                   const uint8_t* mask, cudaStream_t st)
{
    if (src_fp64)
        k_convert_in<double, T><<<elementwise_blocks(n), 256, 0, st>>>((const double*)src, (T*)dst, comp, n, scale,
                                                                       mask);
    else
        k_convert_in<float, T><<<elementwise_blocks(n), 256, 0, st>>>((const float*)src, (T*)dst, comp, n, scale,
                                                                      mask);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::convert_out(const void* src, int comp, void* dst, int dst_fp64, size_t n, double scale,
                                    cudaStream_t st)
{
    if (dst_fp64)
        k_convert_out<T, double><<<elementwise_blocks(n), 256, 0, st>>>((const T*)src, comp, (double*)dst, n, scale);
    else
        k_convert_out<T, float><<<elementwise_blocks(n), 256, 0, st>>>((const T*)src, comp, (float*)dst, n, scale);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::apply_mask(void* q4, const uint8_t* mask, size_t n, cudaStream_t st)
{
    k_apply_mask4<T><<<elementwise_blocks(n), 256, 0, st>>>((T*)q4, mask, n);
    return cudaGetLastError();
}

cudaError_t build_stencil_mask(const uint8_t* mask, uint8_t* smask, int nx, int ny, int nz, cudaStream_t st)
{
    k_build_smask<<<elementwise_blocks((size_t)nx * ny * nz), 256, 0, st>>>(mask, smask, nx, ny, nz);
    return cudaGetLastError();
}

cudaError_t mask_merge(uint8_t* mask, const uint8_t* src, uint8_t bit, size_t n, cudaStream_t st)
{
    k_mask_merge<<<elementwise_blocks(n), 256, 0, st>>>(mask, src, bit, n);
    return cudaGetLastError();
}

cudaError_t mask_fill(uint8_t* mask, uint8_t value, size_t n, cudaStream_t st)
{
    k_mask_fill<<<elementwise_blocks(n), 256, 0, st>>>(mask, value, n);
    return cudaGetLastError();
}

cudaError_t mask_count_solid(const uint8_t* mask, size_t n, unsigned long long* d_count, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_count_solid<<<elementwise_blocks(n), 256, 0, st>>>(mask, n, d_count);
    return cudaGetLastError();
}

cudaError_t mask_mark_near_solid(uint8_t* mask, int nx, int ny, int nz, cudaStream_t st)
{
    k_mark_near_solid<<<elementwise_blocks((size_t)nx * ny * nz), 256, 0, st>>>(mask, nx, ny, nz);
    return cudaGetLastError();
}

cudaError_t mask_mark_budget(uint8_t* mask, int nx, int ny, int nz, cudaStream_t st)
{
    k_mark_budget<<<elementwise_blocks((size_t)nx * ny * nz), 256, 0, st>>>(mask, nx, ny, nz);
    return cudaGetLastError();
}

cudaError_t mask_list_counts(const uint8_t* mask, size_t n, uint8_t bit, int* chunk_counts, cudaStream_t st)
{
    k_list_counts<<<(unsigned)((n + kListChunk - 1) / kListChunk), 256, 0, st>>>(mask, n, bit, chunk_counts);
    return cudaGetLastError();
}

cudaError_t mask_list_fill(const uint8_t* mask, size_t n, uint8_t bit, const int* chunk_offsets, int* list,
                           cudaStream_t st)
{
    k_list_fill<<<(unsigned)((n + kListChunk - 1) / kListChunk), 256, 0, st>>>(mask, n, bit, chunk_offsets, list);
    return cudaGetLastError();
}

template struct Kernels<float>;
template struct Kernels<double>;

}  // namespace vf
