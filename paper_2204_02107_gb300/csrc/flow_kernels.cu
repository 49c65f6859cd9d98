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

#include "vf_internal.h"

namespace vf {
namespace {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int ZCHUNK = 16;   // planes per CTA along z

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
    const int plane = nx * ny;
    const int z0 = blockIdx.z * ZCHUNK;
    const int z1 = min(z0 + ZCHUNK, nz);
    const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
    const int rowc = y * nx, rowm = wrap(y - 1, ny) * nx, rowp = wrap(y + 1, ny) * nx;

    // z registers: the 4-vector and mask at z-1, z, z+1, and the prefetched plane z+2
    T qzm[4], q0[4], qzp[4], qn2[4];
    uint8_t mzm, m0, mzp, mn2 = 0;
    {
        const int im = wrap(z0 - 1, nz) * plane + rowc + x;
        const int ic = z0 * plane + rowc + x;
        const int ip = wrap(z0 + 1, nz) * plane + rowc + x;
        ld4(a.qs, im, qzm);
        ld4(a.qs, ic, q0);
        ld4(a.qs, ip, qzp);
        mzm = __ldg(a.mask + im);
        m0 = __ldg(a.mask + ic);
        mzp = __ldg(a.mask + ip);
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) qn2[f] = T(0);
    for (int z = z0; z < z1; ++z) {
        const int zb = z * plane;
        const int ic = zb + rowc + x;
        if (z + 1 < z1) {   // prefetch plane z+2 for the next iteration
            const int i2 = wrap(z + 2, nz) * plane + rowc + x;
            ld4(a.qs, i2, qn2);
            mn2 = __ldg(a.mask + i2);
        }
        T qm[3][4], qp[3][4];
        ld4(a.qs, zb + rowc + xm, qm[0]);
        ld4(a.qs, zb + rowc + xp, qp[0]);
        ld4(a.qs, zb + rowm + x, qm[1]);
        ld4(a.qs, zb + rowp + x, qp[1]);
#pragma unroll
        for (int f = 0; f < 4; ++f) { qm[2][f] = qzm[f]; qp[2][f] = qzp[f]; }
        T qn[4], ac[4];
        if (STAGE == 2 || STAGE == 3) ld4(a.qn, ic, qn);
        if (STAGE >= 2) ld4(a.acc, ic, ac);   // read by its owner thread before that thread overwrites it
        const uint8_t mxm = __ldg(a.mask + zb + rowc + xm), mxp = __ldg(a.mask + zb + rowc + xp);
        const uint8_t mym = __ldg(a.mask + zb + rowm + x), myp = __ldg(a.mask + zb + rowp + x);
        const T bm[3] = {beta_of<T>(mxm), beta_of<T>(mym), beta_of<T>(mzm)};
        const T bp[3] = {beta_of<T>(mxp), beta_of<T>(myp), beta_of<T>(mzp)};
        const T beta = beta_of<T>(m0);
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
        T o1[4], o2[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            if (STAGE == 1) { o1[f] = q0[f] + k.dt6 * kq[f]; o2[f] = q0[f] + k.dt2 * kq[f]; }
            else if (STAGE == 2) { o1[f] = ac[f] + k.dt3 * kq[f]; o2[f] = qn[f] + k.dt2 * kq[f]; }
            else if (STAGE == 3) { o1[f] = ac[f] + k.dt3 * kq[f]; o2[f] = qn[f] + k.dt * kq[f]; }
            else { o1[f] = T(0); o2[f] = ac[f] + k.dt6 * kq[f]; }
        }
        if (STAGE <= 3) st4(a.acc, ic, o1);
        st4(a.out, ic, o2);
#pragma unroll
        for (int f = 0; f < 4; ++f) { qzm[f] = q0[f]; q0[f] = qzp[f]; qzp[f] = qn2[f]; }
        mzm = m0;
        m0 = mzp;
        mzp = mn2;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Divergence r = sum_j delta_j u_j / dt (a4; divided by dt because the solver works on p / rho)
// ------------------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(TX * TY) k_div(const void* __restrict__ q, T* __restrict__ r, FlowConsts<T> k)
{
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= k.nx || y >= k.ny) return;
    const int nx = k.nx, ny = k.ny, nz = k.nz;
    const int plane = nx * ny;
    const int z0 = blockIdx.z * ZCHUNK, z1 = min(z0 + ZCHUNK, nz);
    const int rowc = y * nx, rowm = wrap(y - 1, ny) * nx, rowp = wrap(y + 1, ny) * nx;
    const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
    T wzm = ld1<T>(q, wrap(z0 - 1, nz) * plane + rowc + x, 2);
    T wz0 = ld1<T>(q, z0 * plane + rowc + x, 2);
    for (int z = z0; z < z1; ++z) {
        const int zb = z * plane;
        const T wzp = ld1<T>(q, wrap(z + 1, nz) * plane + rowc + x, 2);
        const T d = k.i2h_div[0] * (ld1<T>(q, zb + rowc + xp, 0) - ld1<T>(q, zb + rowc + xm, 0)) +
                    k.i2h_div[1] * (ld1<T>(q, zb + rowp + x, 1) - ld1<T>(q, zb + rowm + x, 1)) +
                    k.i2h_div[2] * (wzp - wzm);
        r[zb + rowc + x] = d;
        wzm = wz0;
        wz0 = wzp;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Projection u = beta (u* - dt G p) with p = p / rho (a9); c* passes through.  Ticks the device step counter.
// ------------------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(TX * TY) k_project(const void* __restrict__ qs, const T* __restrict__ p,
                                                     void* __restrict__ out, const uint8_t* __restrict__ mask,
                                                     long long* step_counter, FlowConsts<T> k)
{
    if (step_counter && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
        threadIdx.y == 0)
        *step_counter += 1;
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= k.nx || y >= k.ny) return;
    const int nx = k.nx, ny = k.ny, nz = k.nz;
    const int plane = nx * ny;
    const int z0 = blockIdx.z * ZCHUNK, z1 = min(z0 + ZCHUNK, nz);
    const int rowc = y * nx, rowm = wrap(y - 1, ny) * nx, rowp = wrap(y + 1, ny) * nx;
    const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
    T pzm = __ldg(p + wrap(z0 - 1, nz) * plane + rowc + x);
    T pz0 = __ldg(p + z0 * plane + rowc + x);
    for (int z = z0; z < z1; ++z) {
        const int zb = z * plane;
        const int ic = zb + rowc + x;
        const T pzp = __ldg(p + wrap(z + 1, nz) * plane + rowc + x);
        T q[4];
        ld4(qs, ic, q);
        const T beta = beta_of<T>(__ldg(mask + ic));
        q[0] = beta * (q[0] - k.i2h_dt[0] * (__ldg(p + zb + rowc + xp) - __ldg(p + zb + rowc + xm)));
        q[1] = beta * (q[1] - k.i2h_dt[1] * (__ldg(p + zb + rowp + x) - __ldg(p + zb + rowm + x)));
        q[2] = beta * (q[2] - k.i2h_dt[2] * (pzp - pzm));
        st4(out, ic, q);
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
__global__ void __launch_bounds__(TX * TY) k_filter(const void* __restrict__ in, void* __restrict__ out,
                                                    const uint8_t* __restrict__ mask, FlowConsts<T> k)
{
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    if (x >= k.nx || y >= k.ny) return;
    const int nx = k.nx, ny = k.ny, nz = k.nz;
    const int plane = nx * ny;
    const int z0 = blockIdx.z * ZCHUNK, z1 = min(z0 + ZCHUNK, nz);
    int xo[7], yo[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) {
        xo[m] = wrap(x + m - 3, nx);
        yo[m] = wrap(y + m - 3, ny) * nx;
    }
    // z window of 7 planes of the 4-vector, in registers
    T zw[7][4];
#pragma unroll
    for (int m = 0; m < 6; ++m) ld4(in, wrap(z0 + m - 3, nz) * plane + yo[3] + x, zw[m + 1]);
    for (int z = z0; z < z1; ++z) {
        const int zb = z * plane;
        const int ic = zb + yo[3] + x;
#pragma unroll
        for (int m = 0; m < 6; ++m)
#pragma unroll
            for (int f = 0; f < 4; ++f) zw[m][f] = zw[m + 1][f];
        ld4(in, wrap(z + 3, nz) * plane + yo[3] + x, zw[6]);
        T xn[7][4], yn[7][4];
#pragma unroll
        for (int m = 0; m < 7; ++m) {
            if (m == 3) continue;
            ld4(in, zb + yo[3] + xo[m], xn[m]);
            ld4(in, zb + yo[m] + x, yn[m]);
        }
        const T beta = beta_of<T>(__ldg(mask + ic));
        T o[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const T c = zw[3][f];
            const T sx = s6(xn[0][f], xn[1][f], xn[2][f], c, xn[4][f], xn[5][f], xn[6][f]);
            const T sy = s6(yn[0][f], yn[1][f], yn[2][f], c, yn[4][f], yn[5][f], yn[6][f]);
            const T sz = s6(zw[0][f], zw[1][f], zw[2][f], c, zw[4][f], zw[5][f], zw[6][f]);
            o[f] = beta * (c + k.filt * (sx + sy + sz));
        }
        st4(out, ic, o);
    }
}

// ------------------------------------------------------------------------------------------------------------
// Reductions (a11), one launch.  Each thread sums a z column of ZRED cells; in float it uses compensated
// (TwoSum) additions and the warp combines the (sum, error) pairs as float-float values, so no FP64 arithmetic
// runs per cell.  Each CTA writes one FP64 partial per quantity; the last CTA to finish (atomic ticket) adds
// the partials in CTA order, so the result does not depend on scheduling.  The histogram counts runs of equal
// bins along each column (one shared atomic per run) and adds its CTA counts to global 64-bit counters.
// ------------------------------------------------------------------------------------------------------------
constexpr int ZRED = 16;

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
    // warp-wide sum of the (s, e) pairs, every lane ends with the total
    __device__ double warp_total()
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T s2 = __shfl_xor_sync(0xffffffffu, s, o), e2 = __shfl_xor_sync(0xffffffffu, e, o);
            const T t = s + s2;
            const T bp = t - s;
            e = e + e2 + ((s - (t - bp)) + (s2 - bp));
            s = t;
        }
        return (double)s + (double)e;
    }
};

template <>
struct Acc<double> {
    double s;
    __device__ void init() { s = 0.0; }
    __device__ void add(double v) { s += v; }
    __device__ double warp_total()
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        return s;
    }
};

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename T>
__global__ void __launch_bounds__(TX * TY) k_reduce(const void* __restrict__ q, const uint8_t* __restrict__ mask,
                                                    FlowConsts<T> k, ReduceArgsDev r, int to_history)
{
    constexpr int NW = TX * TY / 32;
    static_assert(NW == kRedSlots, "one warp per reduced quantity in the final pass");
    __shared__ int hist[kHistBins + 2];
    __shared__ long long hist_total[kHistBins + 2];
    __shared__ double red[kRedSlots][NW];
    __shared__ bool is_last;
    const int tid = threadIdx.y * TX + threadIdx.x;
    for (int i = tid; i < kHistBins + 2; i += TX * TY) hist[i] = 0;
    __syncthreads();

    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    Acc<T> ke, d2, ct, cr, c2, vr;
    ke.init(); d2.init(); ct.init(); cr.init(); c2.init(); vr.init();
    T dmax = T(0), umax = T(0);
    bool bad = false;
    int run_bin = -1, run_len = 0;
    if (x < k.nx && y < k.ny) {
        const int nx = k.nx, ny = k.ny, nz = k.nz;
        const int plane = nx * ny;
        const int z0 = blockIdx.z * ZRED, z1 = min(z0 + ZRED, nz);
        const int rowc = y * nx, rowm = wrap(y - 1, ny) * nx, rowp = wrap(y + 1, ny) * nx;
        const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
        T wzm = ld1<T>(q, wrap(z0 - 1, nz) * plane + rowc + x, 2);
        T c4[4];
        ld4(q, z0 * plane + rowc + x, c4);
        for (int z = z0; z < z1; ++z) {
            const int zb = z * plane;
            const int ic = zb + rowc + x;
            T n4[4];
            ld4(q, wrap(z + 1, nz) * plane + rowc + x, n4);
            const T uu = c4[0], vv = c4[1], ww = c4[2], cc = c4[3];
            const T d = k.i2h[0] * (ld1<T>(q, zb + rowc + xp, 0) - ld1<T>(q, zb + rowc + xm, 0)) +
                        k.i2h[1] * (ld1<T>(q, zb + rowp + x, 1) - ld1<T>(q, zb + rowm + x, 1)) +
                        k.i2h[2] * (n4[2] - wzm);
            ke.add(uu * uu + vv * vv + ww * ww);
            d2.add(d * d);
            ct.add(cc);
            dmax = fmax(dmax, fabs(d));
            umax = fmax(umax, fmax(fabs(uu), fmax(fabs(vv), fabs(ww))));
            if (!isfinite(uu) || !isfinite(vv) || !isfinite(ww) || !isfinite(cc)) bad = true;
            if (__ldg(mask + ic) & kBitRoom) {
                cr.add(cc);
                c2.add(cc * cc);
                vr.add(T(1));
                int bin;
                if (cc < T(0)) bin = kHistBins;
                else if (cc > T(1)) bin = kHistBins + 1;
                else bin = min((int)floor(cc * T(kHistBins)), kHistBins - 1);
                if (bin == run_bin) {
                    ++run_len;
                } else {
                    if (run_len) atomicAdd(&hist[run_bin], run_len);
                    run_bin = bin;
                    run_len = 1;
                }
            }
            wzm = ww;
#pragma unroll
            for (int f = 0; f < 4; ++f) c4[f] = n4[f];
        }
    }
    if (run_len) atomicAdd(&hist[run_bin], run_len);
    if (bad) *r.nonfinite = 1;
    const double vals[kRedSlots] = {ke.warp_total(), d2.warp_total(), ct.warp_total(), cr.warp_total(),
                                    c2.warp_total(), vr.warp_total(), warp_max((double)dmax),
                                    warp_max((double)umax)};
    const int lane = tid & 31, wid = tid >> 5;
    if (lane == 0)
#pragma unroll
        for (int qq = 0; qq < kRedSlots; ++qq) red[qq][wid] = vals[qq];
    __syncthreads();
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const long long bid = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    if (tid < kRedSlots) {
        double s = red[tid][0];
        for (int i = 1; i < NW; ++i) s = (tid < 6) ? s + red[tid][i] : fmax(s, red[tid][i]);
        r.partial[bid * kRedSlots + tid] = s;
    }
    for (int i = tid; i < kHistBins + 2; i += TX * TY)
        if (hist[i]) atomicAdd(r.hist_accum + i, (unsigned long long)hist[i]);
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(r.done, 1u) == (unsigned)(nblocks - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // final pass: warp qq adds partial qq of every CTA in CTA order (fixed tree); the histogram counters are read
    // and cleared by one thread each
    {
        const int qq = wid;
        double s = 0.0;
        for (int b = lane; b < nblocks; b += 32) {
            const double pv = __ldcg(r.partial + (long long)b * kRedSlots + qq);
            s = (qq < 6) ? s + pv : fmax(s, pv);
        }
        Acc<double> acc{s};
        s = (qq < 6) ? acc.warp_total() : warp_max(s);
        if (lane == 0) red[qq][0] = s;
    }
    for (int i = tid; i < kHistBins + 2; i += TX * TY) hist_total[i] = (long long)atomicExch(r.hist_accum + i, 0ull);
    __syncthreads();
    // the record is written field by field by several threads (no per-thread copy of the whole struct)
    const long long slot = to_history ? (*r.hist_count % r.history_capacity) : 0;
    vf_reduce* outs[2] = {r.out, to_history ? r.history + slot : nullptr};
    for (int o = 0; o < 2; ++o) {
        vf_reduce* dst = outs[o];
        if (!dst) continue;
        for (int i = tid; i < kHistBins + 2; i += TX * TY) {
            if (i < kHistBins) dst->hist[i] = hist_total[i];
            else if (i == kHistBins) dst->hist_under = hist_total[i];
            else dst->hist_over = hist_total[i];
        }
        if (tid == 0) {
            const long long step = *r.step_counter;
            dst->step = step;
            dst->t = r.t0 + (double)step * r.dt;
            dst->ke = 0.5 * r.dV * red[0][0];
            dst->div_l2 = sqrt(r.dV * red[1][0]);
            dst->c_total = r.dV * red[2][0];
            dst->c_room = r.dV * red[3][0];
            dst->c2_room = r.dV * red[4][0];
            dst->v_room = r.dV * red[5][0];
            dst->div_max = red[6][0];
            dst->u_max = red[7][0];
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (!isfinite(red[0][0]) || !isfinite(red[2][0])) *r.nonfinite = 1;
        if (to_history) *r.hist_count += 1;
        *r.done = 0u;
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

__global__ void k_near_counts(const uint8_t* __restrict__ mask, size_t n, int* counts)
{
    __shared__ int warp_tot[kListChunk / 32];
    const size_t base = (size_t)blockIdx.x * kListChunk;
    int local = 0;
    for (int t = threadIdx.x; t < kListChunk; t += blockDim.x) {
        const size_t i = base + t;
        if (i < n && (mask[i] & kBitNearSolid)) ++local;
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
__global__ void k_near_fill(const uint8_t* __restrict__ mask, size_t n, const int* __restrict__ offsets, int* list)
{
    __shared__ int warp_tot[32];
    __shared__ int running;
    const size_t base = (size_t)blockIdx.x * kListChunk;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) running = offsets[blockIdx.x];
    __syncthreads();
    for (int r = 0; r < kListChunk; r += blockDim.x) {
        const size_t i = base + r + threadIdx.x;
        const bool flag = i < n && (mask[i] & kBitNearSolid);
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

inline dim3 flow_grid(int nx, int ny, int nz)
{
    return dim3((nx + TX - 1) / TX, (ny + TY - 1) / TY, (nz + ZCHUNK - 1) / ZCHUNK);
}

inline dim3 reduce_grid(int nx, int ny, int nz)
{
    return dim3((nx + TX - 1) / TX, (ny + TY - 1) / TY, (nz + ZRED - 1) / ZRED);
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
cudaError_t Kernels<T>::divergence(const void* qstar, T* r, const FlowConsts<T>& k, cudaStream_t st)
{
    k_div<T><<<flow_grid(k.nx, k.ny, k.nz), dim3(TX, TY), 0, st>>>(qstar, r, k);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::project(const void* qstar, const T* p, void* out, const uint8_t* mask,
                                long long* step_counter, const FlowConsts<T>& k, cudaStream_t st)
{
    k_project<T><<<flow_grid(k.nx, k.ny, k.nz), dim3(TX, TY), 0, st>>>(qstar, p, out, mask, step_counter, k);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Kernels<T>::filter(const void* in, void* out, const uint8_t* mask, const FlowConsts<T>& k,
                               cudaStream_t st)
{
    k_filter<T><<<flow_grid(k.nx, k.ny, k.nz), dim3(TX, TY), 0, st>>>(in, out, mask, k);
    return cudaGetLastError();
}

template <typename T>
int Kernels<T>::reduce_blocks(const FlowConsts<T>& k)
{
    const dim3 g = reduce_grid(k.nx, k.ny, k.nz);
    return (int)(g.x * g.y * g.z);
}

template <typename T>
cudaError_t Kernels<T>::reduce(const void* q, const uint8_t* mask, const FlowConsts<T>& k, const ReduceArgsDev& r,
                               int to_history, cudaStream_t st)
{
    k_reduce<T><<<reduce_grid(k.nx, k.ny, k.nz), dim3(TX, TY), 0, st>>>(q, mask, k, r, to_history);
    return cudaGetLastError();
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

cudaError_t mask_near_counts(const uint8_t* mask, size_t n, int* chunk_counts, cudaStream_t st)
{
    k_near_counts<<<(unsigned)((n + kListChunk - 1) / kListChunk), 256, 0, st>>>(mask, n, chunk_counts);
    return cudaGetLastError();
}

cudaError_t mask_near_fill(const uint8_t* mask, size_t n, const int* chunk_offsets, int* list, cudaStream_t st)
{
    k_near_fill<<<(unsigned)((n + kListChunk - 1) / kListChunk), 256, 0, st>>>(mask, n, chunk_offsets, list);
    return cudaGetLastError();
}

template struct Kernels<float>;
template struct Kernels<double>;

}  // namespace vf
