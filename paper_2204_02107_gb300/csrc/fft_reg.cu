// Register-resident passes of the FFT Poisson solve (Sec. 2.2, Eqs. 7-9) for grids whose axis lengths are all
// 16 G with G in {1, 2, 4, 8, 16} (nx = 32 G_x); the (y, z) work is one whole-plane kernel when the plane of one kx
// fits in shared memory, else the tile mode further down.
//
// A transform of n = 16 G points is done by G threads of one warp.  Thread t holds x[t + G m] (m = 0..15),
// does a 16-point DFT in registers, multiplies by W_n^(t k1), exchanges through a slice of shared memory that
// only its group touches (so a __syncwarp orders the exchange, never a CTA barrier), and finishes with 16 / G
// DFTs of order G.  It then holds X[t Q + q + 16 k2] (Q = 16 / G) in register q G + k2.  The inverse is the
// mirror image and ends with thread t holding x[t + G m] again, so global loads and stores stay coalesced.
//
// One iteration of Eq. 9 is the correction (masked grids) and three kernels (five when the plane of one kx does not
// fit in shared memory: the (y, z) kernel becomes a y pass, a z pass over tiles of y slots, and an inverse y pass):
//   x forward : real-to-complex FFT along x of f (r plus the Eq. 9 correction, added beforehand at the cells
//               next to solids by the correction kernel of the generic path), two reals packed per complex
//               value, split step written straight into the plane layout spec[kx][z][y] (the rows of a warp
//               are consecutive, so every frequency is one contiguous piece of at least 32 bytes);
//   (y, z)    : one CTA per kx plane: y FFT of every z row straight from global memory into the shared plane,
//               z FFT of every column, division by lambda N, inverse z FFT (one register pass per column),
//               inverse y FFT back to global memory;
//   x inverse : each warp gathers its rows from the plane layout, joins, inverse FFT, writes p^{k+1}.
// The arithmetic (DFT kernels, twiddle tables, packing, eigenvalues) is the one of the generic passes; only the
// order of the butterflies and the data movement differ.
#include <algorithm>
#include <cstdlib>

#include "fft_common.cuh"

namespace vf {
namespace {

template <int G>
struct RegShape {
    static constexpr int Q = 16 / G;
    // exchange slot of the k1-th 16-point output of thread t (skewed so both sides of the exchange spread over
    // the shared-memory banks)
    static __device__ __forceinline__ int xpos(int t, int k1) { return k1 * G + ((t + k1 / Q) & (G - 1)); }
    // slot and frequency of held value (q, k2) of thread t
    static __device__ __forceinline__ int slot(int t, int q, int k2) { return t + G * q + 16 * k2; }
    static __device__ __forceinline__ int freq(int t, int q, int k2) { return t * Q + q + 16 * k2; }
};

// slot of frequency k (the inverse of RegShape::freq followed by RegShape::slot)
template <int G>
__device__ __forceinline__ int slot_of_freq(int k)
{
    constexpr int Q = 16 / G;
    const int k1 = k & 15, k2 = k >> 4;
    return (k1 / Q) + G * (k1 % Q) + 16 * k2;
}

// frequency held at slot s
template <int G>
__device__ __forceinline__ int freq_of_slot(int s)
{
    constexpr int Q = 16 / G;
    const int r = s & 15, k2 = s >> 4;
    return (r % G) * Q + r / G + 16 * k2;
}

// forward transform of v (thread t of its group); buf(e) is element e of the group's exchange slice
template <typename C, int G, typename BUF>
__device__ __forceinline__ void reg_fwd(C v[16], int t, const C* tw, BUF buf)
{
    dft<C, 16, false>(v);
    if constexpr (G > 1) {
        constexpr int Q = 16 / G;
#pragma unroll
        for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], tw[t * k1]);
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) buf(RegShape<G>::xpos(t, k1)) = v[k1];
        __syncwarp();
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int s = 0; s < G; ++s) v[q * G + s] = buf(RegShape<G>::xpos(s, t * Q + q));
#pragma unroll
        for (int q = 0; q < Q; ++q) dft<C, G, false>(v + q * G);
    }
}

// inverse transform (unnormalised) from the held layout back to v[m] = n x[t + G m]
template <typename C, int G, typename BUF>
__device__ __forceinline__ void reg_inv(C v[16], int t, const C* tw, BUF buf)
{
    if constexpr (G > 1) {
        constexpr int Q = 16 / G;
#pragma unroll
        for (int q = 0; q < Q; ++q) dft<C, G, true>(v + q * G);
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int s = 1; s < G; ++s) {
                C w = tw[s * (t * Q + q)];
                w.y = -w.y;
                v[q * G + s] = cmul(v[q * G + s], w);
            }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int s = 0; s < G; ++s) buf(RegShape<G>::xpos(s, t * Q + q)) = v[q * G + s];
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) v[k1] = buf(RegShape<G>::xpos(t, k1));
    }
    dft<C, 16, true>(v);
}

// x passes: 128-thread CTAs in both precisions (FP32: 1024 CTAs over 8 per SM balance the SMs better than 512 over
// 4, measured 12.5 / 12.4 vs 12.8 / 13.3 us per pass on the 256 x 128 x 128 room)
template <typename T> __host__ __device__ constexpr int x_threads() { return 128; }
// (y, z) plane kernel: 512 threads in FP32 (up to 128 registers a thread; with 1024 threads the 64-register cap
// spills the transforms: 15.7 against 18.2 us per launch on the 256 x 128 x 128 room)
#ifndef VF_REG_YZ_THREADS
#define VF_REG_YZ_THREADS 512
#endif
template <typename T> __host__ __device__ constexpr int yz_threads() { return sizeof(T) == 4 ? VF_REG_YZ_THREADS : 512; }

// ---- x forward ---------------------------------------------------------------------------------------------
// Each warp works alone on its 32 / GX rows: the split step writes X_k of its rows straight to the plane layout
// spec[k][row] (the rows of a warp are consecutive, so each frequency is one contiguous 32-byte or longer piece).
template <typename T, int GX>
__global__ void __launch_bounds__(x_threads<T>()) k_reg_x_fwd(PoissonArgs<T> A)
{
    pdl_enter();
    using C = typename CxT<T>::type;
    constexpr int M = 16 * GX, NT = x_threads<T>(), B = NT / GX, P = 32 / GX, Q = 16 / GX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int SPX = A.reg_spx;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* twr = tw + M;
    C* rowbuf = twr + (M + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane % P, t = lane / P;
    const int b = warp * P + gi;
    const int rows = A.ny * A.nz, row = blockIdx.x * B + b;
    const bool act = row < rows;
    C v[16];
    {   // the row's loads are issued before the tables are staged
        const T* __restrict__ src = A.f + (long long)(act ? row : 0) * A.nx;
#pragma unroll
        for (int m = 0; m < 16; ++m)
            v[m] = act ? *reinterpret_cast<const C*>(src + 2 * (t + GX * m)) : mk<C>(T(0), T(0));
    }
    stage_table(tw, A.twx, M);
    stage_table(twr, A.twr, M + 1);
    __syncthreads();
    C* rb = rowbuf + b * SPX;
    auto buf = [rb](int e) -> C& { return rb[e]; };
    reg_fwd<C, GX>(v, t, tw, buf);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int k2 = 0; k2 < GX; ++k2) rb[RegShape<GX>::slot(t, q, k2)] = v[q * GX + k2];
    __syncwarp();
    // the split results go straight to the plane layout (rows of a warp are consecutive), or, for rows of 256
    // frequencies (two rows per warp, 16-byte pieces), through a frequency-major stage so that each frequency of
    // the CTA's B rows leaves as one contiguous piece
    constexpr bool STAGED = GX == 16;
    constexpr int SB = B + 1;
    C* stage = rowbuf + B * SPX;
    C* __restrict__ spec = reinterpret_cast<C*>(A.spec) + (act ? row : 0);
    auto put = [&](int k, C val) {
        if (STAGED) stage[k * SB + b] = val;
        else if (act) spec[(long long)k * rows] = val;
    };
    // split step: X_k = E_k + W^k O_k from Z_k and conj Z_{M-k}; the pair (k, M - k) by one thread,
    // k = t + GX i for i = 0..8 (k = M / 2 only for t = 0)
#pragma unroll
    for (int i = 0; i <= 8; ++i) {
        const int k = t + GX * i;
        if (k > M / 2) break;
        const C Zk = rb[slot_of_freq<GX>(k)];
        if (k == 0) {
            put(0, mk<C>(Zk.x + Zk.y, Zk.x - Zk.y));                  // (X_0, X_{nx/2})
            continue;
        }
        const C Zm = rb[slot_of_freq<GX>(M - k)];
        {
            const C E = mk<C>(T(0.5) * (Zk.x + Zm.x), T(0.5) * (Zk.y - Zm.y));
            const C O = mk<C>(T(0.5) * (Zk.y + Zm.y), T(-0.5) * (Zk.x - Zm.x));
            put(k, cadd(E, cmul(twr[k], O)));
        }
        if (2 * k != M) {
            const C E = mk<C>(T(0.5) * (Zm.x + Zk.x), T(0.5) * (Zm.y - Zk.y));
            const C O = mk<C>(T(0.5) * (Zm.y + Zk.y), T(-0.5) * (Zm.x - Zk.x));
            put(M - k, cadd(E, cmul(twr[M - k], O)));
        }
    }
    if (STAGED) {
        __syncthreads();
        C* out = reinterpret_cast<C*>(A.spec);
        const int row0 = blockIdx.x * B;
        for (int it = threadIdx.x; it < M * B; it += NT) {
            const int k = it / B, bb = it - k * B;
            if (row0 + bb < rows) out[(long long)k * rows + row0 + bb] = stage[k * SB + bb];
        }
    }
}

// ---- x inverse ---------------------------------------------------------------------------------------------
template <typename T, int GX>
__global__ void __launch_bounds__(x_threads<T>()) k_reg_x_inv(PoissonArgs<T> A)
{
    pdl_enter();
    using C = typename CxT<T>::type;
    constexpr int M = 16 * GX, NT = x_threads<T>(), B = NT / GX, P = 32 / GX, Q = 16 / GX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int SPX = A.reg_spx;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* twr = tw + M;
    C* rowbuf = twr + (M + 1);
    stage_table(tw, A.twx, M);
    stage_table(twr, A.twr, M + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane % P, t = lane / P;
    const int b = warp * P + gi;
    const int rows = A.ny * A.nz, row = blockIdx.x * B + b;
    const bool act = row < rows;
    // the pairs (X_k, X_{M-k}) of this thread, k = t + GX i: straight from the plane layout with all loads in
    // flight together, or (rows of 256 frequencies) gathered first for the CTA's B rows into a frequency-major stage
    constexpr bool STAGED = GX == 16;
    constexpr int SB = B + 1;
    C* stage = rowbuf + B * SPX;
    C xk[9], xm[9];
    if (STAGED) {
        const C* __restrict__ in = reinterpret_cast<const C*>(A.spec);
        const int row0 = blockIdx.x * B;
        for (int it0 = threadIdx.x; it0 < M * B; it0 += 8 * NT) {
            C tmp[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int it = it0 + u * NT, k = it / B, bb = it - k * B;
                tmp[u] = (it < M * B && row0 + bb < rows) ? in[(long long)k * rows + row0 + bb] : mk<C>(T(0), T(0));
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int it = it0 + u * NT, k = it / B, bb = it - k * B;
                if (it < M * B) stage[k * SB + bb] = tmp[u];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i <= 8; ++i) {
            const int k = t + GX * i;
            const bool ok = k <= M / 2;
            xk[i] = ok ? stage[k * SB + b] : mk<C>(T(0), T(0));
            xm[i] = ok && k > 0 ? stage[(M - k) * SB + b] : mk<C>(T(0), T(0));
        }
    } else {
        const C* __restrict__ spec = reinterpret_cast<const C*>(A.spec) + (act ? row : 0);
#pragma unroll
        for (int i = 0; i <= 8; ++i) {
            const int k = t + GX * i;
            const bool ok = act && k <= M / 2;
            xk[i] = ok ? spec[(long long)k * rows] : mk<C>(T(0), T(0));
            xm[i] = ok && k > 0 ? spec[(long long)(M - k) * rows] : mk<C>(T(0), T(0));
        }
        __syncthreads();   // tables staged
    }
    C* rb = rowbuf + b * SPX;
    // join: Z'_k = (X_k + conj X_{M-k}) + i W^{-k} (X_k - conj X_{M-k})
#pragma unroll
    for (int i = 0; i <= 8; ++i) {
        const int k = t + GX * i;
        if (k > M / 2) break;
        const C Xk = xk[i], Xm = xm[i];
        if (k == 0) {
            rb[slot_of_freq<GX>(0)] = mk<C>(Xk.x + Xk.y, Xk.x - Xk.y);
            continue;
        }
        {
            const C s = mk<C>(Xk.x + Xm.x, Xk.y - Xm.y), d = mk<C>(Xk.x - Xm.x, Xk.y + Xm.y);
            C w = twr[k];
            w.y = -w.y;
            const C wd = cmul(w, d);
            rb[slot_of_freq<GX>(k)] = mk<C>(s.x - wd.y, s.y + wd.x);
        }
        if (2 * k != M) {
            const C s = mk<C>(Xm.x + Xk.x, Xm.y - Xk.y), d = mk<C>(Xm.x - Xk.x, Xm.y + Xk.y);
            C w = twr[M - k];
            w.y = -w.y;
            const C wd = cmul(w, d);
            rb[slot_of_freq<GX>(M - k)] = mk<C>(s.x - wd.y, s.y + wd.x);
        }
    }
    __syncwarp();
    C v[16];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int k2 = 0; k2 < GX; ++k2) v[q * GX + k2] = rb[RegShape<GX>::slot(t, q, k2)];
    auto buf = [rb](int e) -> C& { return rb[e]; };
    reg_inv<C, GX>(v, t, tw, buf);
    if (act) {
        T* __restrict__ dst = A.p + (long long)row * A.nx;
#pragma unroll
        for (int m = 0; m < 16; ++m) *reinterpret_cast<C*>(dst + 2 * (t + GX * m)) = v[m];
    }
}

// ---- (y, z) plane of one kx ----------------------------------------------------------------------------------
template <typename T, int GY, int GZ>
__global__ void __launch_bounds__(yz_threads<T>()) k_reg_yz_solve(PoissonArgs<T> A)
{
    pdl_enter();
    using C = typename CxT<T>::type;
    constexpr int NY = 16 * GY, NZ = 16 * GZ, QY = 16 / GY, QZ = 16 / GZ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int SP = A.reg_sp;
    C* plane = reinterpret_cast<C*>(smem_raw);     // row z at z * SP, slot s of the y transform at s
    C* twy = plane + NZ * SP;
    C* twz = twy + NY;
    stage_table(twy, A.twy, NY);
    stage_table(twz, A.twz, NZ);
    const int kx = blockIdx.x;
    C* g = reinterpret_cast<C*>(A.spec) + (long long)kx * NY * NZ;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    // y forward: a group per z row, global memory -> registers -> shared plane (slots)
    {
        constexpr int P = 32 / GY;
        const int gi = lane % P, t = lane / P;
        for (int z0 = warp * P; z0 < NZ; z0 += nwarps * P) {
            const int z = z0 + gi;
            const bool act = z < NZ;             // false only for G = 1 with NZ = 16 (no exchange then)
            C v[16];
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = act ? g[z * NY + t + GY * m] : mk<C>(T(0), T(0));
            C* row = plane + (act ? z : 0) * SP;
            auto buf = [row](int e) -> C& { return row[e]; };
            reg_fwd<C, GY>(v, t, twy, buf);
            __syncwarp();
            if (act) {
#pragma unroll
                for (int q = 0; q < QY; ++q)
#pragma unroll
                    for (int k2 = 0; k2 < GY; ++k2) row[RegShape<GY>::slot(t, q, k2)] = v[q * GY + k2];
            }
        }
    }
    __syncthreads();
    // z: a group per column (y slot c): forward FFT, x 1 / (lambda N), inverse FFT, in place in the column
    {
        constexpr int P = 32 / GZ;
        const int gi = lane % P, t = lane / P;
        const T lx = __ldg(A.lamx + kx);
        for (int c0 = warp * P; c0 < NY; c0 += nwarps * P) {
            const int c = c0 + gi;
            const bool act = c < NY;
            const int cc = act ? c : 0;
            const int ky = freq_of_slot<GY>(cc);
            const T lxy = lx + __ldg(A.lamy + ky);
            const bool ky_null = (kx == 0) && (ky == 0 || 2 * ky == NY);
            C v[16];
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = plane[(t + GZ * m) * SP + cc];
            auto buf = [plane, SP, cc](int e) -> C& { return plane[e * SP + cc]; };
            reg_fwd<C, GZ>(v, t, twz, buf);
#pragma unroll
            for (int q = 0; q < QZ; ++q)
#pragma unroll
                for (int k2 = 0; k2 < GZ; ++k2) {
                    const int kz = RegShape<GZ>::freq(t, q, k2);
                    const bool null = ky_null && (kz == 0 || 2 * kz == NZ);
                    const T s = null ? T(0) : inv_lambda(A.invN, lxy + __ldg(A.lamz + kz));
                    v[q * GZ + k2] = cscale(v[q * GZ + k2], s);
                }
            reg_inv<C, GZ>(v, t, twz, buf);
            __syncwarp();
            if (act) {
#pragma unroll
                for (int m = 0; m < 16; ++m) plane[(t + GZ * m) * SP + cc] = v[m];
            }
        }
    }
    __syncthreads();
    // y inverse: a group per z row, shared plane -> registers -> global memory
    {
        constexpr int P = 32 / GY;
        const int gi = lane % P, t = lane / P;
        for (int z0 = warp * P; z0 < NZ; z0 += nwarps * P) {
            const int z = z0 + gi;
            const bool act = z < NZ;
            C* row = plane + (act ? z : 0) * SP;
            C v[16];
#pragma unroll
            for (int q = 0; q < QY; ++q)
#pragma unroll
                for (int k2 = 0; k2 < GY; ++k2) v[q * GY + k2] = row[RegShape<GY>::slot(t, q, k2)];
            auto buf = [row](int e) -> C& { return row[e]; };
            reg_inv<C, GY>(v, t, twy, buf);
            if (act) {
#pragma unroll
                for (int m = 0; m < 16; ++m) g[z * NY + t + GY * m] = v[m];
            }
        }
    }
}

// ---- tile mode: the (y, z) plane of one kx does not fit in shared memory ----------------------------------------
// ky held at y slot s after the forward y pass (run-time G)
__device__ __forceinline__ int freq_of_slot_rt(int s, int g)
{
    const int r = s & 15, k2 = s >> 4;
    return (r % g) * (16 / g) + r / g + 16 * k2;
}

// y pass: a group per spectrum row (kx, z), straight from and to global memory.  The forward pass leaves the y
// spectrum of a row in slot order (ky of slot s is freq_of_slot), which the z pass reads and the inverse pass
// takes back to natural order.
template <typename T, int GY, bool INV>
__global__ void __launch_bounds__(256) k_reg_y(PoissonArgs<T> A)
{
    pdl_enter();
    using C = typename CxT<T>::type;
    constexpr int NY = 16 * GY, B = 256 / GY, P = 32 / GY, Q = 16 / GY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int SY = A.reg_sy;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* rowbuf = tw + NY;
    stage_table(tw, A.twy, NY);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane % P, t = lane / P;
    const int b = warp * P + gi;
    const long long rows = (long long)A.M * A.nz;
    const long long row = (long long)blockIdx.x * B + b;
    const bool act = row < rows;
    C* g = reinterpret_cast<C*>(A.spec) + (act ? row : 0) * NY;
    C* rb = rowbuf + b * SY;
    auto buf = [rb](int e) -> C& { return rb[e]; };
    C v[16];
    if (!INV) {
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = act ? g[t + GY * m] : mk<C>(T(0), T(0));
        reg_fwd<C, GY>(v, t, tw, buf);
        if (act) {
#pragma unroll
            for (int q = 0; q < Q; ++q)
#pragma unroll
                for (int k2 = 0; k2 < GY; ++k2) g[RegShape<GY>::slot(t, q, k2)] = v[q * GY + k2];
        }
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int k2 = 0; k2 < GY; ++k2)
                v[q * GY + k2] = act ? g[RegShape<GY>::slot(t, q, k2)] : mk<C>(T(0), T(0));
        reg_inv<C, GY>(v, t, tw, buf);
        if (act) {
#pragma unroll
            for (int m = 0; m < 16; ++m) g[t + GY * m] = v[m];
        }
    }
}

// z pass: a CTA takes TB consecutive y slots of one kx plane and all z, staged as a shared tile [z][slot] with
// coalesced loads; a group per column does the forward z FFT, the division by lambda N and the inverse z FFT in
// registers, then the tile goes back.
#ifndef VF_ZTILE_MIN_CTAS
#define VF_ZTILE_MIN_CTAS 4
#endif
template <typename T, int GZ>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? VF_ZTILE_MIN_CTAS : 2) k_reg_z_tile(PoissonArgs<T> A)
{
    pdl_enter();
    using C = typename CxT<T>::type;
    constexpr int NZ = 16 * GZ, P = 32 / GZ, QZ = 16 / GZ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ST = A.reg_st, TB = A.reg_tb, ny = A.ny;
    C* tile = reinterpret_cast<C*>(smem_raw);     // element (z, c) at z * ST + c
    C* twz = tile + (size_t)NZ * ST;
    const int tiles = ny / TB;
    const int tb_shift = __ffs(TB) - 1;          // TB is a power of two
    const int kx = blockIdx.x / tiles, c0 = (blockIdx.x - kx * tiles) * TB;
    C* g = reinterpret_cast<C*>(A.spec) + (long long)kx * ny * NZ;
    const int n_el = NZ * TB, nt = blockDim.x;
    for (int i0 = threadIdx.x; i0 < n_el; i0 += 8 * nt) {
        C tmp[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * nt;
            if (i < n_el) {
                const int z = i >> tb_shift, c = i & (TB - 1);
                tmp[u] = g[(long long)z * ny + c0 + c];
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * nt;
            if (i < n_el) {
                const int z = i >> tb_shift, c = i & (TB - 1);
                tile[z * ST + c] = tmp[u];
            }
        }
    }
    stage_table(twz, A.twz, NZ);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = lane % P, t = lane / P;
    const int c = warp * P + gi;                  // blockDim = TB * GZ: every group has a column
    const int ky = freq_of_slot_rt(c0 + c, A.gy);
    const T lxy = __ldg(A.lamx + kx) + __ldg(A.lamy + ky);
    const bool ky_null = (kx == 0) && (ky == 0 || 2 * ky == ny);
    C v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = tile[(t + GZ * m) * ST + c];
    auto buf = [tile, ST, c](int e) -> C& { return tile[e * ST + c]; };
    reg_fwd<C, GZ>(v, t, twz, buf);
#pragma unroll
    for (int q = 0; q < QZ; ++q)
#pragma unroll
        for (int k2 = 0; k2 < GZ; ++k2) {
            const int kz = RegShape<GZ>::freq(t, q, k2);
            const bool null = ky_null && (kz == 0 || 2 * kz == NZ);
            const T s = null ? T(0) : inv_lambda(A.invN, lxy + __ldg(A.lamz + kz));
            v[q * GZ + k2] = cscale(v[q * GZ + k2], s);
        }
    reg_inv<C, GZ>(v, t, twz, buf);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 16; ++m) tile[(t + GZ * m) * ST + c] = v[m];
    __syncthreads();
    for (int i0 = threadIdx.x; i0 < n_el; i0 += 8 * nt) {
        C tmp[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * nt;
            if (i < n_el) {
                const int z = i >> tb_shift, cc = i & (TB - 1);
                tmp[u] = tile[z * ST + cc];
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * nt;
            if (i < n_el) {
                const int z = i >> tb_shift, cc = i & (TB - 1);
                g[(long long)z * ny + c0 + cc] = tmp[u];
            }
        }
    }
}

// ---- host side ---------------------------------------------------------------------------------------------
int g_of(int n)
{
    for (int g = 1; g <= 16; g *= 2)
        if (n == 16 * g) return g;
    return 0;
}

// Worst number of distinct 8-byte words one bank serves in a warp access (shared memory: 16 banks of 8 bytes
// per 128-byte wavefront for 8-byte elements, 32 of 4 bytes = 16 of 8).  addr(lane, step) in elements of esz bytes.
template <typename F>
int worst_ways(int esz, F addr)
{
    int worst = 1;
    for (int step = 0; step < 16; ++step) {
        int ways[32] = {0};
        long long seen[32][32];
        int nseen[32] = {0};
        for (int lane = 0; lane < 32; ++lane) {
            const long long byte = addr(lane, step) * (long long)esz;
            for (int w = 0; w < esz / 4; ++w) {
                const long long word = byte / 4 + w;
                const int bank = (int)(word % 32);
                bool dup = false;
                for (int i = 0; i < nseen[bank]; ++i) dup |= seen[bank][i] == word;
                if (!dup && nseen[bank] < 32) { seen[bank][nseen[bank]++] = word; ways[bank]++; }
            }
        }
        for (int i = 0; i < 32; ++i) worst = ways[i] > worst ? ways[i] : worst;
    }
    return worst;
}

int xpos_h(int G, int t, int k1) { const int Q = 16 / G; return k1 * G + ((t + k1 / Q) & (G - 1)); }

// conflicts of the row-owned accesses (a group of G threads per row, rows `stride` apart)
int row_ways(int G, int stride, int esz)
{
    const int P = 32 / G, Q = 16 / G;
    int w = 0;
    auto mx = [&](int v) { w = v > w ? v : w; };
    if (G > 1) {
        mx(worst_ways(esz, [&](int l, int s) { return (long long)(l % P) * stride + xpos_h(G, l / P, s); }));
        mx(worst_ways(esz, [&](int l, int s) {
            return (long long)(l % P) * stride + xpos_h(G, s % G, (l / P) * Q + (s / G) % Q); }));
    }
    mx(worst_ways(esz, [&](int l, int s) { return (long long)(l % P) * stride + (l / P) + G * (s % Q) + 16 * ((s / Q) % G); }));
    return w;
}

// conflicts of the column-owned accesses (element e of column c at e * stride + c)
int col_ways(int G, int stride, int esz)
{
    const int P = 32 / G, Q = 16 / G;
    int w = 0;
    auto mx = [&](int v) { w = v > w ? v : w; };
    mx(worst_ways(esz, [&](int l, int s) { return (long long)((l / P) + G * s) * stride + (l % P); }));
    if (G > 1) {
        mx(worst_ways(esz, [&](int l, int s) { return (long long)xpos_h(G, l / P, s) * stride + (l % P); }));
        mx(worst_ways(esz, [&](int l, int s) {
            return (long long)xpos_h(G, s % G, (l / P) * Q + (s / G) % Q) * stride + (l % P); }));
    }
    return w;
}

template <typename T>
size_t x_smem(int M, int spx)
{
    const int B = x_threads<T>() / (M / 16);
    const size_t stage = M == 256 ? (size_t)M * (B + 1) : 0;     // the frequency-major stage of 256-point rows
    return ((size_t)M + (M + 1) + (size_t)B * spx + stage) * sizeof(typename CxT<T>::type);
}

template <typename T>
size_t yz_smem(int ny, int nz, int sp)
{
    return ((size_t)nz * sp + ny + nz) * sizeof(typename CxT<T>::type);
}

template <typename T>
size_t y_smem(int ny, int sy)
{
    const int B = 256 / (ny / 16);
    return ((size_t)ny + (size_t)B * sy) * sizeof(typename CxT<T>::type);
}

template <typename T>
size_t ztile_smem(int nz, int st)
{
    return ((size_t)nz * st + nz) * sizeof(typename CxT<T>::type);
}

constexpr size_t kRegSmemLimit = 200 * 1024;

template <typename T, int GY>
cudaError_t launch_y(const PoissonArgs<T>& a, bool inv, cudaStream_t st)
{
    constexpr int B = 256 / GY;
    const long long rows = (long long)a.M * a.nz;
    const unsigned grid = (unsigned)((rows + B - 1) / B);
    const size_t sm = y_smem<T>(16 * GY, a.reg_sy);
    return launch_pdl(inv ? k_reg_y<T, GY, true> : k_reg_y<T, GY, false>, dim3(grid), dim3(256), sm, st, a);
}

template <typename T>
cudaError_t dispatch_y(const PoissonArgs<T>& a, bool inv, cudaStream_t st)
{
    switch (a.gy) {
        case 1: return launch_y<T, 1>(a, inv, st);
        case 2: return launch_y<T, 2>(a, inv, st);
        case 4: return launch_y<T, 4>(a, inv, st);
        case 8: return launch_y<T, 8>(a, inv, st);
        case 16: return launch_y<T, 16>(a, inv, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int GZ>
cudaError_t launch_ztile(const PoissonArgs<T>& a, cudaStream_t st)
{
    const unsigned grid = (unsigned)(a.M * (a.ny / a.reg_tb));
    return launch_pdl(k_reg_z_tile<T, GZ>, dim3(grid), dim3(a.reg_tb * GZ), ztile_smem<T>(16 * GZ, a.reg_st), st, a);
}

template <typename T>
cudaError_t dispatch_ztile(const PoissonArgs<T>& a, cudaStream_t st)
{
    switch (a.gz) {
        case 1: return launch_ztile<T, 1>(a, st);
        case 2: return launch_ztile<T, 2>(a, st);
        case 4: return launch_ztile<T, 4>(a, st);
        case 8: return launch_ztile<T, 8>(a, st);
        case 16: return launch_ztile<T, 16>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int GX>
cudaError_t launch_x(const PoissonArgs<T>& a, bool fwd, cudaStream_t st)
{
    constexpr int B = x_threads<T>() / GX;
    const int rows = a.ny * a.nz;
    const unsigned grid = (unsigned)((rows + B - 1) / B);
    const size_t sm = x_smem<T>(16 * GX, a.reg_spx);
    return launch_pdl(fwd ? k_reg_x_fwd<T, GX> : k_reg_x_inv<T, GX>, dim3(grid), dim3(x_threads<T>()), sm, st, a);
}

template <typename T>
cudaError_t dispatch_x(const PoissonArgs<T>& a, bool fwd, cudaStream_t st)
{
    switch (a.gx) {
        case 1: return launch_x<T, 1>(a, fwd, st);
        case 2: return launch_x<T, 2>(a, fwd, st);
        case 4: return launch_x<T, 4>(a, fwd, st);
        case 8: return launch_x<T, 8>(a, fwd, st);
        case 16: return launch_x<T, 16>(a, fwd, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int GY, int GZ>
cudaError_t launch_yz(const PoissonArgs<T>& a, cudaStream_t st)
{
    const int want = (16 * GY) * (16 * GZ) / 16;
    const int threads = want < 32 ? 32 : (want > yz_threads<T>() ? yz_threads<T>() : want);
    return launch_pdl(k_reg_yz_solve<T, GY, GZ>, dim3(a.M), dim3(threads), yz_smem<T>(a.ny, a.nz, a.reg_sp), st, a);
}

template <typename T, int GY>
cudaError_t dispatch_yz_z(const PoissonArgs<T>& a, cudaStream_t st)
{
    switch (a.gz) {
        case 1: return launch_yz<T, GY, 1>(a, st);
        case 2: return launch_yz<T, GY, 2>(a, st);
        case 4: return launch_yz<T, GY, 4>(a, st);
        case 8: return launch_yz<T, GY, 8>(a, st);
        case 16: return launch_yz<T, GY, 16>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t dispatch_yz(const PoissonArgs<T>& a, cudaStream_t st)
{
    switch (a.gy) {
        case 1: return dispatch_yz_z<T, 1>(a, st);
        case 2: return dispatch_yz_z<T, 2>(a, st);
        case 4: return dispatch_yz_z<T, 4>(a, st);
        case 8: return dispatch_yz_z<T, 8>(a, st);
        case 16: return dispatch_yz_z<T, 16>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename K>
cudaError_t raise_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (bytes > (size_t)optin) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

template <typename T, int GX>
cudaError_t prepare_x(const PoissonArgs<T>& a)
{
    const size_t sm = x_smem<T>(16 * GX, a.reg_spx);
    cudaError_t e = raise_smem(k_reg_x_fwd<T, GX>, sm);
    if (e == cudaSuccess) e = raise_smem(k_reg_x_inv<T, GX>, sm);
    return e;
}

template <typename T, int G>
cudaError_t prepare_tile(const PoissonArgs<T>& a)
{
    // y passes of length 16 G and the z tile of length 16 G (each used when its axis has this G)
    cudaError_t e = cudaSuccess;
    if (a.gy == G) {
        const size_t sm = y_smem<T>(16 * G, a.reg_sy);
        e = raise_smem(k_reg_y<T, G, false>, sm);
        if (e == cudaSuccess) e = raise_smem(k_reg_y<T, G, true>, sm);
    }
    if (e == cudaSuccess && a.gz == G) e = raise_smem(k_reg_z_tile<T, G>, ztile_smem<T>(16 * G, a.reg_st));
    return e;
}

template <typename T, int GY>
cudaError_t prepare_yz_z(const PoissonArgs<T>& a)
{
    const size_t sm = yz_smem<T>(a.ny, a.nz, a.reg_sp);
    switch (a.gz) {
        case 1: return raise_smem(k_reg_yz_solve<T, GY, 1>, sm);
        case 2: return raise_smem(k_reg_yz_solve<T, GY, 2>, sm);
        case 4: return raise_smem(k_reg_yz_solve<T, GY, 4>, sm);
        case 8: return raise_smem(k_reg_yz_solve<T, GY, 8>, sm);
        case 16: return raise_smem(k_reg_yz_solve<T, GY, 16>, sm);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

template <typename T>
bool RegFft<T>::eligible(int nx, int ny, int nz)
{
    if (nx % 2) return false;
    const int gx = g_of(nx / 2), gy = g_of(ny), gz = g_of(nz);
    if (!gx || !gy || !gz) return false;
    // the x passes must fit; the (y, z) plane goes through shared memory whole when it fits, else in tiles
    return x_smem<T>(nx / 2, nx / 2 + 15) <= kRegSmemLimit && y_smem<T>(ny, ny + 15) <= kRegSmemLimit;
}

template <typename T>
void RegFft<T>::configure(PoissonArgs<T>& a)
{
    a.reg = 0;
    if (!eligible(a.nx, a.ny, a.nz)) return;
    a.gx = g_of(a.M);
    a.gy = g_of(a.ny);
    a.gz = g_of(a.nz);
    const int esz = (int)sizeof(typename CxT<T>::type);
    // plane stride: fewest bank conflicts over the y-row and z-column accesses, then the smallest
    int best = -1, best_w = 1 << 30;
    for (int pad = 0; pad < 16; ++pad) {
        const int sp = a.ny + pad;
        const int w = std::max(row_ways(a.gy, sp, esz), col_ways(a.gz, sp, esz));
        if (w < best_w) { best_w = w; best = sp; }
    }
    a.reg_sp = best;
    a.reg_tile = (yz_smem<T>(a.ny, a.nz, a.reg_sp) > kRegSmemLimit || std::getenv("VF_REG_TILE")) ? 1 : 0;
    if (a.reg_tile) {
        // y passes: the row slices of the groups; z tile: TB slots of one plane, columns as for the plane
        best = -1; best_w = 1 << 30;
        for (int pad = 0; pad < 16; ++pad) {
            const int w = row_ways(a.gy, a.ny + pad, esz);
            if (w < best_w) { best_w = w; best = a.ny + pad; }
        }
        a.reg_sy = best;
        a.reg_tb = std::min(a.ny, 256 / a.gz);
        best = -1; best_w = 1 << 30;
        for (int pad = 0; pad < 16; ++pad) {
            const int w = col_ways(a.gz, a.reg_tb + pad, esz);
            if (w < best_w) { best_w = w; best = a.reg_tb + pad; }
        }
        a.reg_st = best;
    }
    // x passes: the row slices of the groups
    best = -1; best_w = 1 << 30;
    for (int pad = 0; pad < 16; ++pad) {
        const int w = row_ways(a.gx, a.M + pad, esz);
        if (w < best_w) { best_w = w; best = a.M + pad; }
    }
    a.reg_spx = best;
    a.reg_sb = 0;
    a.reg = 1;
}

template <typename T>
cudaError_t RegFft<T>::prepare(const PoissonArgs<T>& a)
{
    if (!a.reg) return cudaErrorInvalidValue;
    cudaError_t e;
    switch (a.gx) {
        case 1: e = prepare_x<T, 1>(a); break;
        case 2: e = prepare_x<T, 2>(a); break;
        case 4: e = prepare_x<T, 4>(a); break;
        case 8: e = prepare_x<T, 8>(a); break;
        case 16: e = prepare_x<T, 16>(a); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (a.reg_tile) {
        if ((e = prepare_tile<T, 1>(a)) != cudaSuccess) return e;
        if ((e = prepare_tile<T, 2>(a)) != cudaSuccess) return e;
        if ((e = prepare_tile<T, 4>(a)) != cudaSuccess) return e;
        if ((e = prepare_tile<T, 8>(a)) != cudaSuccess) return e;
        return prepare_tile<T, 16>(a);
    }
    switch (a.gy) {
        case 1: return prepare_yz_z<T, 1>(a);
        case 2: return prepare_yz_z<T, 2>(a);
        case 4: return prepare_yz_z<T, 4>(a);
        case 8: return prepare_yz_z<T, 8>(a);
        case 16: return prepare_yz_z<T, 16>(a);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t RegFft<T>::iteration(const PoissonArgs<T>& a, cudaStream_t st, const LaunchHook* hook)
{
    if (!a.reg) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = dispatch_x<T>(a, true, st)) != cudaSuccess) return e;
    if (hook) (*hook)(VF_PHASE_FFT_X_FWD);
    if (a.reg_tile) {
        if ((e = dispatch_y<T>(a, false, st)) != cudaSuccess) return e;
        if (hook) (*hook)(VF_PHASE_FFT_Y_FWD);
        if ((e = dispatch_ztile<T>(a, st)) != cudaSuccess) return e;
        if (hook) (*hook)(VF_PHASE_FFT_Z_SOLVE);
        if ((e = dispatch_y<T>(a, true, st)) != cudaSuccess) return e;
        if (hook) (*hook)(VF_PHASE_FFT_Y_INV);
    } else {
        if ((e = dispatch_yz<T>(a, st)) != cudaSuccess) return e;
        if (hook) (*hook)(VF_PHASE_FFT_YZ_SOLVE);
    }
    if ((e = dispatch_x<T>(a, false, st)) != cudaSuccess) return e;
    if (hook) (*hook)(VF_PHASE_FFT_X_INV);
    return cudaSuccess;
}

template struct RegFft<float>;
template struct RegFft<double>;

}  // namespace vf
