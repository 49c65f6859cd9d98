// Flow kernels of the DNSLABIB time step (Sec. 2.1-2.2): fused RK4 stages, divergence, projection, sixth-order
// filter, FP64 reductions, and the small conversion / mask kernels behind the C ABI.
//
// Layout: one array per field, x fastest (index x + nx*(y + ny*z)), periodic in all three directions.  A CTA
// covers a 32 x 8 (x, y) tile and marches along z, keeping the centre column of every field in registers so that
// each plane is loaded from global memory once (the z neighbours come from the registers of the previous and
// next iteration; the x and y neighbours come through L1).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "vf_internal.h"

namespace vf {
namespace {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int ZCHUNK = 16;   // planes per CTA along z

struct Nbr {
    long long c, xm, xp, ym, yp;   // centre and in-plane neighbours of the current plane
};

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <typename T>
__device__ __forceinline__ T ld(const T* p, long long i) { return __ldg(p + i); }

__device__ __forceinline__ float beta_of(uint8_t m, float) { return (m & kBitBeta) ? 1.0f : 0.0f; }
__device__ __forceinline__ double beta_of(uint8_t m, double) { return (m & kBitBeta) ? 1.0 : 0.0; }

// ------------------------------------------------------------------------------------------------------------
// RK4 stage (a1 + a2 + a3)
// ------------------------------------------------------------------------------------------------------------
// k_i = beta [ -sum_j q4h_j ((U_j Q_i)^+ - (U_j Q_i)^- + U_j^0 (Q_i^+ - Q_i^-))          (skew convection)
//              + nu sum_j ih2_j (Q_i^+ - 2 Q_i^0 + Q_i^-)                                  (diffusion)
//              + S (uset_i - Q_i^0) inv_tau + b_i ]                                        (forcing, body force)
// k_c = beta [ -sum_j ih_j (F^+ - F^-) + alpha sum_j ih2_j (beta^+ (c^+ - c^0) - beta^- (c^0 - c^-))
//              + S (cset - c^0) inv_tau ],  F^+ = beta^+ (U_j^0 c^0 + U_j^+ c^+) / 2 (face weight beta^0 beta^+,
//              beta^0 is applied by the outer factor)
template <typename T, int STAGE>
__global__ void __launch_bounds__(TX * TY) k_stage(StageArgs<T> a, FlowConsts<T> k)
{
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= k.nx || y >= k.ny) return;
    const int nx = k.nx, ny = k.ny, nz = k.nz;
    const long long plane = (long long)nx * ny;
    const int z0 = blockIdx.z * ZCHUNK;
    const int z1 = min(z0 + ZCHUNK, nz);
    const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
    const int ym = wrap(y - 1, ny), yp = wrap(y + 1, ny);
    const long long rowc = (long long)y * nx, rowm = (long long)ym * nx, rowp = (long long)yp * nx;

    // z-neighbour registers: values of the 4 fields and the mask at z-1, z, z+1 in this column
    T qzm[4], q0[4], qzp[4];
    uint8_t mzm, m0, mzp;
    {
        const long long im = (long long)wrap(z0 - 1, nz) * plane + rowc + x;
        const long long ic = (long long)z0 * plane + rowc + x;
#pragma unroll
        for (int f = 0; f < 4; ++f) { qzm[f] = ld(a.qs[f], im); q0[f] = ld(a.qs[f], ic); }
        mzm = __ldg(a.mask + im);
        m0 = __ldg(a.mask + ic);
    }
    for (int z = z0; z < z1; ++z) {
        const long long zb = (long long)z * plane;
        const long long ic = zb + rowc + x;
        const long long izp = (long long)wrap(z + 1, nz) * plane + rowc + x;
#pragma unroll
        for (int f = 0; f < 4; ++f) qzp[f] = ld(a.qs[f], izp);
        mzp = __ldg(a.mask + izp);

        const long long ixm = zb + rowc + xm, ixp = zb + rowc + xp;
        const long long iym = zb + rowm + x, iyp = zb + rowp + x;
        T qm[3][4], qp[3][4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            qm[0][f] = ld(a.qs[f], ixm); qp[0][f] = ld(a.qs[f], ixp);
            qm[1][f] = ld(a.qs[f], iym); qp[1][f] = ld(a.qs[f], iyp);
            qm[2][f] = qzm[f];           qp[2][f] = qzp[f];
        }
        const uint8_t mxm = __ldg(a.mask + ixm), mxp = __ldg(a.mask + ixp);
        const uint8_t mym = __ldg(a.mask + iym), myp = __ldg(a.mask + iyp);
        const T bm[3] = {beta_of(mxm, T()), beta_of(mym, T()), beta_of(mzm, T())};
        const T bp[3] = {beta_of(mxp, T()), beta_of(myp, T()), beta_of(mzp, T())};
        const T beta = beta_of(m0, T());
        const T S = (m0 & kBitS) ? T(1) : T(0);

        T kq[4];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            T conv = T(0), diff = T(0);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                conv += k.q4h[j] * ((qp[j][j] * qp[j][i] - qm[j][j] * qm[j][i]) + q0[j] * (qp[j][i] - qm[j][i]));
                diff += k.ih2[j] * (qp[j][i] - T(2) * q0[i] + qm[j][i]);
            }
            kq[i] = beta * (-conv + k.nu * diff + S * (k.uset[i] - q0[i]) * k.inv_tau + k.bf[i]);
        }
        {
            const T c0 = q0[3];
            T conv = T(0), diff = T(0);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const T uc0 = q0[j] * c0;
                const T Fp = bp[j] * T(0.5) * (uc0 + qp[j][j] * qp[j][3]);
                const T Fm = bm[j] * T(0.5) * (qm[j][j] * qm[j][3] + uc0);
                conv += k.ih[j] * (Fp - Fm);
                diff += k.ih2[j] * (bp[j] * (qp[j][3] - c0) - bm[j] * (c0 - qm[j][3]));
            }
            kq[3] = beta * (-conv + k.alpha * diff + S * (k.cset - c0) * k.inv_tau);
        }

        // RK4 combine (classic tableau: nodes 0, 1/2, 1/2, 1; weights 1/6, 1/3, 1/3, 1/6)
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            if (STAGE == 1) {
                const T qn = q0[f];
                a.acc[f][ic] = qn + k.dt6 * kq[f];
                a.out[f][ic] = qn + k.dt2 * kq[f];
            } else if (STAGE == 2) {
                const T qn = ld(a.qn[f], ic);
                a.acc[f][ic] = a.acc[f][ic] + k.dt3 * kq[f];
                a.out[f][ic] = qn + k.dt2 * kq[f];
            } else if (STAGE == 3) {
                const T qn = ld(a.qn[f], ic);
                a.acc[f][ic] = a.acc[f][ic] + k.dt3 * kq[f];
                a.out[f][ic] = qn + k.dt * kq[f];
            } else {
                a.out[f][ic] = a.acc[f][ic] + k.dt6 * kq[f];
            }
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) { qzm[f] = q0[f]; q0[f] = qzp[f]; }
        mzm = m0;
        m0 = mzp;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Divergence r = sum_j delta_j u_j / dt (a4; divided by dt because the solver works on p / rho)
// ------------------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(TX * TY) k_div(const T* __restrict__ u, const T* __restrict__ v,
                                                 const T* __restrict__ w, T* __restrict__ r, FlowConsts<T> k)
{
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= k.nx || y >= k.ny) return;
    const int nx = k.nx, ny = k.ny, nz = k.nz;
    const long long plane = (long long)nx * ny;
    const int z0 = blockIdx.z * ZCHUNK, z1 = min(z0 + ZCHUNK, nz);
    const long long rowc = (long long)y * nx;
    const long long rowm = (long long)wrap(y - 1, ny) * nx, rowp = (long long)wrap(y + 1, ny) * nx;
    const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
    T wzm = ld(w, (long long)wrap(z0 - 1, nz) * plane + rowc + x);
    T wz0 = ld(w, (long long)z0 * plane + rowc + x);
    for (int z = z0; z < z1; ++z) {
        const long long zb = (long long)z * plane;
        const T wzp = ld(w, (long long)wrap(z + 1, nz) * plane + rowc + x);
        const T d = k.i2h_div[0] * (ld(u, zb + rowc + xp) - ld(u, zb + rowc + xm)) +
                    k.i2h_div[1] * (ld(v, zb + rowp + x) - ld(v, zb + rowm + x)) + k.i2h_div[2] * (wzp - wzm);
        r[zb + rowc + x] = d;
        wzm = wz0;
        wz0 = wzp;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Projection u = beta (u* - dt G p) with p = p / rho (a9); also carries c* to its output and ticks the device
// step counter
// ------------------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(TX * TY) k_project(const T* __restrict__ us, const T* __restrict__ vs,
                                                     const T* __restrict__ ws, const T* __restrict__ cs,
                                                     const T* __restrict__ p, T* __restrict__ uo, T* __restrict__ vo,
                                                     T* __restrict__ wo, T* __restrict__ co,
                                                     const uint8_t* __restrict__ mask, long long* step_counter,
                                                     FlowConsts<T> k)
{
    if (step_counter && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
        threadIdx.y == 0)
        *step_counter += 1;
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= k.nx || y >= k.ny) return;
    const int nx = k.nx, ny = k.ny, nz = k.nz;
    const long long plane = (long long)nx * ny;
    const int z0 = blockIdx.z * ZCHUNK, z1 = min(z0 + ZCHUNK, nz);
    const long long rowc = (long long)y * nx;
    const long long rowm = (long long)wrap(y - 1, ny) * nx, rowp = (long long)wrap(y + 1, ny) * nx;
    const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
    T pzm = ld(p, (long long)wrap(z0 - 1, nz) * plane + rowc + x);
    T pz0 = ld(p, (long long)z0 * plane + rowc + x);
    for (int z = z0; z < z1; ++z) {
        const long long zb = (long long)z * plane;
        const long long ic = zb + rowc + x;
        const T pzp = ld(p, (long long)wrap(z + 1, nz) * plane + rowc + x);
        const T beta = beta_of(__ldg(mask + ic), T());
        uo[ic] = beta * (ld(us, ic) - k.i2h_dt[0] * (ld(p, zb + rowc + xp) - ld(p, zb + rowc + xm)));
        vo[ic] = beta * (ld(vs, ic) - k.i2h_dt[1] * (ld(p, zb + rowp + x) - ld(p, zb + rowm + x)));
        wo[ic] = beta * (ld(ws, ic) - k.i2h_dt[2] * (pzp - pzm));
        if (co != cs) co[ic] = ld(cs, ic);
        pzm = pz0;
        pz0 = pzp;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Sixth-order filter q <- beta (q + pi^-6 sum_j S6_j q), S6 = (1, -6, 15, -20, 15, -6, 1) (a10, Eq. 6)
// ------------------------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T s6(T m3, T m2, T m1, T c, T p1, T p2, T p3)
{
    return (m3 + p3) - T(6) * (m2 + p2) + T(15) * (m1 + p1) - T(20) * c;
}

template <typename T>
__global__ void __launch_bounds__(TX * TY) k_filter(const T* __restrict__ in0, const T* __restrict__ in1,
                                                    const T* __restrict__ in2, const T* __restrict__ in3,
                                                    T* __restrict__ o0, T* __restrict__ o1, T* __restrict__ o2,
                                                    T* __restrict__ o3, const uint8_t* __restrict__ mask,
                                                    FlowConsts<T> k)
{
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= k.nx || y >= k.ny) return;
    const int nx = k.nx, ny = k.ny, nz = k.nz;
    const long long plane = (long long)nx * ny;
    const int z0 = blockIdx.z * ZCHUNK, z1 = min(z0 + ZCHUNK, nz);
    int xo[7];
    long long yo[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) {
        xo[m] = wrap(x + m - 3, nx);
        yo[m] = (long long)wrap(y + m - 3, ny) * nx;
    }
    const T* in[4] = {in0, in1, in2, in3};
    T* out[4] = {o0, o1, o2, o3};
    // z window of 7 planes for each field, in registers
    T zw[4][7];
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int m = 0; m < 6; ++m) zw[f][m + 1] = ld(in[f], (long long)wrap(z0 + m - 3, nz) * plane + yo[3] + x);
    for (int z = z0; z < z1; ++z) {
        const long long zb = (long long)z * plane;
        const long long ic = zb + yo[3] + x;
        const long long izn = (long long)wrap(z + 3, nz) * plane + yo[3] + x;
        const T beta = beta_of(__ldg(mask + ic), T());
#pragma unroll
        for (int f = 0; f < 4; ++f) {
#pragma unroll
            for (int m = 0; m < 6; ++m) zw[f][m] = zw[f][m + 1];
            zw[f][6] = ld(in[f], izn);
            const T* q = in[f];
            const T c = zw[f][3];
            const T sx = s6(ld(q, zb + yo[3] + xo[0]), ld(q, zb + yo[3] + xo[1]), ld(q, zb + yo[3] + xo[2]), c,
                            ld(q, zb + yo[3] + xo[4]), ld(q, zb + yo[3] + xo[5]), ld(q, zb + yo[3] + xo[6]));
            const T sy = s6(ld(q, zb + yo[0] + x), ld(q, zb + yo[1] + x), ld(q, zb + yo[2] + x), c,
                            ld(q, zb + yo[4] + x), ld(q, zb + yo[5] + x), ld(q, zb + yo[6] + x));
            const T sz = s6(zw[f][0], zw[f][1], zw[f][2], c, zw[f][4], zw[f][5], zw[f][6]);
            out[f][ic] = beta * (c + k.filt * (sx + sy + sz));
        }
    }
}

// ------------------------------------------------------------------------------------------------------------
// Reductions (a11): per-CTA partials in FP64, then one CTA sums them in a fixed order (deterministic).
// In float, each thread first sums its z column with compensated (TwoSum) float additions.
// ------------------------------------------------------------------------------------------------------------
template <typename T>
struct Acc {
    T s, e;   // running sum and its compensation
    __device__ void init() { s = T(0); e = T(0); }
    __device__ void add(T v)
    {
        const T t = s + v;
        const T bp = t - s;
        e += (s - (t - bp)) + (v - bp);
        s = t;
    }
    __device__ double value() const { return (double)s + (double)e; }
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename T>
__global__ void __launch_bounds__(TX * TY) k_reduce(const T* __restrict__ u, const T* __restrict__ v,
                                                    const T* __restrict__ w, const T* __restrict__ c,
                                                    const uint8_t* __restrict__ mask, FlowConsts<T> k,
                                                    ReduceArgsDev r)
{
    __shared__ int hist[kHistBins + 2];
    __shared__ double red[kRedSlots][TX * TY / 32];
    const int tid = threadIdx.y * TX + threadIdx.x;
    for (int i = tid; i < kHistBins + 2; i += TX * TY) hist[i] = 0;
    __syncthreads();

    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    Acc<T> ke, d2, ct, cr, c2, vr;
    ke.init(); d2.init(); ct.init(); cr.init(); c2.init(); vr.init();
    T dmax = T(0), umax = T(0);
    bool bad = false;
    if (x < k.nx && y < k.ny) {
        const int nx = k.nx, ny = k.ny, nz = k.nz;
        const long long plane = (long long)nx * ny;
        const int z0 = blockIdx.z * ZCHUNK, z1 = min(z0 + ZCHUNK, nz);
        const long long rowc = (long long)y * nx;
        const long long rowm = (long long)wrap(y - 1, ny) * nx, rowp = (long long)wrap(y + 1, ny) * nx;
        const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
        T wzm = ld(w, (long long)wrap(z0 - 1, nz) * plane + rowc + x);
        T wz0 = ld(w, (long long)z0 * plane + rowc + x);
        for (int z = z0; z < z1; ++z) {
            const long long zb = (long long)z * plane;
            const long long ic = zb + rowc + x;
            const T wzp = ld(w, (long long)wrap(z + 1, nz) * plane + rowc + x);
            const T uu = ld(u, ic), vv = ld(v, ic), cc = ld(c, ic);
            const T d = k.i2h[0] * (ld(u, zb + rowc + xp) - ld(u, zb + rowc + xm)) +
                        k.i2h[1] * (ld(v, zb + rowp + x) - ld(v, zb + rowm + x)) + k.i2h[2] * (wzp - wzm);
            ke.add(uu * uu + vv * vv + wz0 * wz0);
            d2.add(d * d);
            ct.add(cc);
            dmax = fmax(dmax, fabs(d));
            umax = fmax(umax, fmax(fabs(uu), fmax(fabs(vv), fabs(wz0))));
            if (!isfinite(uu) || !isfinite(vv) || !isfinite(wz0) || !isfinite(cc)) bad = true;
            if (__ldg(mask + ic) & kBitRoom) {
                cr.add(cc);
                c2.add(cc * cc);
                vr.add(T(1));
                int bin;
                if (cc < T(0)) bin = kHistBins;
                else if (cc > T(1)) bin = kHistBins + 1;
                else bin = min((int)floor(cc * T(kHistBins)), kHistBins - 1);
                atomicAdd(&hist[bin], 1);
            }
            wzm = wz0;
            wz0 = wzp;
        }
    }
    if (bad) *r.nonfinite = 1;
    double vals[kRedSlots] = {ke.value(), d2.value(), ct.value(), cr.value(), c2.value(), vr.value(),
                              (double)dmax, (double)umax};
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int q = 0; q < kRedSlots; ++q) {
        const double s = (q < 6) ? warp_sum(vals[q]) : warp_max(vals[q]);
        if (lane == 0) red[q][wid] = s;
    }
    __syncthreads();
    const long long bid = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    if (tid < kRedSlots) {
        double s = red[tid][0];
        for (int i = 1; i < TX * TY / 32; ++i) s = (tid < 6) ? s + red[tid][i] : fmax(s, red[tid][i]);
        r.partial[bid * kRedSlots + tid] = s;
    }
    for (int i = tid; i < kHistBins + 2; i += TX * TY) r.hist_partial[bid * (kHistBins + 2) + i] = hist[i];
}

__global__ void __launch_bounds__(256) k_reduce_final(ReduceArgsDev r, int nblocks, int to_history)
{
    __shared__ double sh[kRedSlots][256];
    __shared__ long long hs[kHistBins + 2];
    const int tid = threadIdx.x;
    double acc[kRedSlots];
#pragma unroll
    for (int q = 0; q < kRedSlots; ++q) acc[q] = 0.0;
    for (int b = tid; b < nblocks; b += 256) {
#pragma unroll
        for (int q = 0; q < kRedSlots; ++q) {
            const double v = r.partial[(long long)b * kRedSlots + q];
            acc[q] = (q < 6) ? acc[q] + v : fmax(acc[q], v);
        }
    }
#pragma unroll
    for (int q = 0; q < kRedSlots; ++q) sh[q][tid] = acc[q];
    for (int i = tid; i < kHistBins + 2; i += 256) {
        long long s = 0;
        for (int b = 0; b < nblocks; ++b) s += r.hist_partial[(long long)b * (kHistBins + 2) + i];
        hs[i] = s;
    }
    __syncthreads();
    for (int stride = 128; stride > 0; stride >>= 1) {
        if (tid < stride) {
#pragma unroll
            for (int q = 0; q < kRedSlots; ++q)
                sh[q][tid] = (q < 6) ? sh[q][tid] + sh[q][tid + stride] : fmax(sh[q][tid], sh[q][tid + stride]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        vf_reduce o;
        const long long step = *r.step_counter;
        o.step = step;
        o.t = r.t0 + (double)step * r.dt;
        o.ke = 0.5 * r.dV * sh[0][0];
        o.div_l2 = sqrt(r.dV * sh[1][0]);
        o.c_total = r.dV * sh[2][0];
        o.c_room = r.dV * sh[3][0];
        o.c2_room = r.dV * sh[4][0];
        o.v_room = r.dV * sh[5][0];
        o.div_max = sh[6][0];
        o.u_max = sh[7][0];
        for (int i = 0; i < kHistBins; ++i) o.hist[i] = hs[i];
        o.hist_under = hs[kHistBins];
        o.hist_over = hs[kHistBins + 1];
        if (!isfinite(o.ke) || !isfinite(o.c_total)) *r.nonfinite = 1;
        *r.out = o;
        if (to_history) {
            const long long n = *r.hist_count;
            r.history[n % r.history_capacity] = o;
            *r.hist_count = n + 1;
        }
    }
}

// ------------------------------------------------------------------------------------------------------------
// Conversions and masks
// ------------------------------------------------------------------------------------------------------------
template <typename Tin, typename Tout>
__global__ void k_convert(const Tin* __restrict__ src, Tout* __restrict__ dst, size_t n, double scale,
                          const uint8_t* __restrict__ mask)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double v = (double)src[i] * scale;
        if (mask && !(mask[i] & kBitBeta)) v = 0.0;
        dst[i] = (Tout)v;
    }
}

template <typename T>
__global__ void k_apply_mask(T* f, const uint8_t* __restrict__ mask, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(mask[i] & kBitBeta)) f[i] = T(0);
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

inline dim3 flow_grid(int nx, int ny, int nz)
{
    return dim3((nx + TX - 1) / TX, (ny + TY - 1) / TY, (nz + ZCHUNK - 1) / ZCHUNK);
}

inline int elementwise_blocks(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

}  // namespace

// ------------------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------------------
template <typename T>
cudaError_t Kernels<T>::stage(int s, const StageArgs<T>& a, const FlowConsts<T>& k, cudaStream_t st)
{
    const dim3 g = flow_grid(k.nx, k.ny, k.nz), b(TX, TY);
    switch (s) {
        case 1: k_stage<T, 1><<<g, b, 0, st>>>(a, k); break;
        case 2: k_stage<T, 2><<<g, b, 0, st>>>(a, k); break;
        case 3: k_stage<T, 3><<<g, b, 0, st>>>(a, k); break;
        case 4: k_stage<T, 4><<<g, b, 0, st>>>(a, k); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::divergence(const T* u, const T* v, const T* w, T* r, const FlowConsts<T>& k,
                                   cudaStream_t st)
{
    k_div<T><<<flow_grid(k.nx, k.ny, k.nz), dim3(TX, TY), 0, st>>>(u, v, w, r, k);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::project(const T* const us[3], const T* cs, const T* p, T* const out[4],
                                const uint8_t* mask, long long* step_counter, const FlowConsts<T>& k,
                                cudaStream_t st)
{
    k_project<T><<<flow_grid(k.nx, k.ny, k.nz), dim3(TX, TY), 0, st>>>(us[0], us[1], us[2], cs, p, out[0], out[1],
                                                                       out[2], out[3], mask, step_counter, k);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::filter(const T* const in[4], T* const out[4], const uint8_t* mask, const FlowConsts<T>& k,
                               cudaStream_t st)
{
    k_filter<T><<<flow_grid(k.nx, k.ny, k.nz), dim3(TX, TY), 0, st>>>(in[0], in[1], in[2], in[3], out[0], out[1],
                                                                      out[2], out[3], mask, k);
    return cudaGetLastError();
}

template <typename T>
int Kernels<T>::reduce_blocks(const FlowConsts<T>& k)
{
    const dim3 g = flow_grid(k.nx, k.ny, k.nz);
    return (int)(g.x * g.y * g.z);
}

template <typename T>
cudaError_t Kernels<T>::reduce(const T* const q[4], const uint8_t* mask, const FlowConsts<T>& k,
                               const ReduceArgsDev& r, int to_history, cudaStream_t st)
{
    k_reduce<T><<<flow_grid(k.nx, k.ny, k.nz), dim3(TX, TY), 0, st>>>(q[0], q[1], q[2], q[3], mask, k, r);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, 256, 0, st>>>(r, reduce_blocks(k), to_history);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::convert_in(const void* src, int src_fp64, T* dst, size_t n, double scale,
                                   const uint8_t* mask, cudaStream_t st)
{
    if (src_fp64)
        k_convert<double, T><<<elementwise_blocks(n), 256, 0, st>>>((const double*)src, dst, n, scale, mask);
    else
        k_convert<float, T><<<elementwise_blocks(n), 256, 0, st>>>((const float*)src, dst, n, scale, mask);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::convert_out(const T* src, void* dst, int dst_fp64, size_t n, double scale, cudaStream_t st)
{
    if (dst_fp64)
        k_convert<T, double><<<elementwise_blocks(n), 256, 0, st>>>(src, (double*)dst, n, scale, nullptr);
    else
        k_convert<T, float><<<elementwise_blocks(n), 256, 0, st>>>(src, (float*)dst, n, scale, nullptr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::apply_mask(T* f, const uint8_t* mask, size_t n, cudaStream_t st)
{
    k_apply_mask<T><<<elementwise_blocks(n), 256, 0, st>>>(f, mask, n);
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

template struct Kernels<float>;
template struct Kernels<double>;

}  // namespace vf
