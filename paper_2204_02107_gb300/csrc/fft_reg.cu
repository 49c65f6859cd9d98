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

// Shape of a register transform of n = R G points: G threads (a power of two dividing 32) hold R values each for
// the first stage, then Q = ceil(R / G) second-stage transforms of order G each, those of k1 = t Q + q.  Where G
// does not divide R the last transforms of a thread may lie past R: they run on zeros and are not stored.
template <int R, int G>
struct RegShape {
    static_assert(32 % G == 0, "a transform's G threads lie in one warp");
    static constexpr int Q = (R + G - 1) / G;
    static constexpr bool EVEN = R % G == 0;
    static constexpr int V = Q * G;   // values a thread holds after the exchange (R when G divides R)
    // exchange slot of the k1-th R-point output of thread t (skewed so both sides of the exchange spread over
    // the shared-memory banks)
    static __device__ __forceinline__ int xpos(int t, int k1) { return k1 * G + ((t + k1 / Q) & (G - 1)); }
    // held value (q, k2) of thread t is a frequency (k1 = t Q + q < R)
    static __device__ __forceinline__ bool valid(int t, int q) { return EVEN || t * Q + q < R; }
    // slot and frequency of held value (q, k2) of thread t (slots in frequency order where G does not divide R)
    static __device__ __forceinline__ int slot(int t, int q, int k2) { return EVEN ? t + G * q + R * k2 : t * Q + q + R * k2; }
    static __device__ __forceinline__ int freq(int t, int q, int k2) { return t * Q + q + R * k2; }
};

// Lanes of a warp split into 32 / G groups of G threads: for G = 4 a group's threads are adjacent lanes, else lane
// i of group g is lane g + i 32 / G.  Shared memory serves an 8-byte access by half-warps (16-byte: by quarters),
// each 128 bytes; with its threads adjacent, a 4-thread group's four consecutive elements and the next rows' lie
// in one half-warp, which a row stride of 4 mod 16 elements spreads over all banks (the host's bank model picks
// the stride for the mapping in use).
template <int G> __host__ __device__ constexpr bool adjacent_groups() { return G == 4; }
template <int G> __device__ __forceinline__ int group_of(int lane) { return adjacent_groups<G>() ? lane / G : lane % (32 / G); }
template <int G> __device__ __forceinline__ int member_of(int lane) { return adjacent_groups<G>() ? lane % G : lane / (32 / G); }

// slot of frequency k (the inverse of RegShape::freq followed by RegShape::slot)
template <int R, int G>
__device__ __forceinline__ int slot_of_freq(int k)
{
    if constexpr (!RegShape<R, G>::EVEN) return k;
    constexpr int Q = R / G;
    const int k1 = k % R, k2 = k / R;
    return (k1 / Q) + G * (k1 % Q) + R * k2;
}

// frequency held at slot s
template <int R, int G>
__device__ __forceinline__ int freq_of_slot(int s)
{
    if constexpr (!RegShape<R, G>::EVEN) return s;
    constexpr int Q = R / G;
    const int r = s % R, k2 = s / R;
    return (r % G) * Q + r / G + R * k2;
}

// forward transform of v[0 .. R) (thread t of its group) into the held layout v[0 .. V); buf(e) is element e of the
// group's exchange slice
template <typename C, int R, int G, typename BUF>
__device__ __forceinline__ void reg_fwd(C* v, int t, const C* tw, BUF buf)
{
    dft<C, R, false>(v);
    if constexpr (G > 1) {
        using S = RegShape<R, G>;
        constexpr int Q = S::Q;
#pragma unroll
        for (int k1 = 1; k1 < R; ++k1) v[k1] = cmul(v[k1], tw[t * k1]);
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) buf(S::xpos(t, k1)) = v[k1];
        __syncwarp();
        C zero;
        zero.x = zero.y = decltype(zero.x)(0);
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int s = 0; s < G; ++s) v[q * G + s] = S::valid(t, q) ? buf(S::xpos(s, t * Q + q)) : zero;
#pragma unroll
        for (int q = 0; q < Q; ++q) dft<C, G, false>(v + q * G);
    }
}

// inverse transform (unnormalised) from the held layout v[0 .. V) back to v[m] = n x[t + G m], m < R
template <typename C, int R, int G, typename BUF>
__device__ __forceinline__ void reg_inv(C* v, int t, const C* tw, BUF buf)
{
    if constexpr (G > 1) {
        using S = RegShape<R, G>;
        constexpr int Q = S::Q;
#pragma unroll
        for (int q = 0; q < Q; ++q) dft<C, G, true>(v + q * G);
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int s = 1; s < G; ++s) {
                if (!S::valid(t, q)) continue;
                C w = tw[s * (t * Q + q)];
                w.y = -w.y;
                v[q * G + s] = cmul(v[q * G + s], w);
            }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int s = 0; s < G; ++s)
                if (S::valid(t, q)) buf(S::xpos(s, t * Q + q)) = v[q * G + s];
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) v[k1] = buf(S::xpos(t, k1));
    }
    dft<C, R, true>(v);
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
// threads of the plane kernel: one pass over the y rows (NZ groups of GY) and the z columns (NY groups of GZ),
// at most yz_threads for lengths 16 G; the 2-3-5 planes (at most 384 threads) take exactly one pass, so that the
// transforms of 18 .. 36 values a thread have up to 255 registers
template <typename T, int RY, int GY, int RZ, int GZ>
__host__ __device__ constexpr int yz_nt()
{
    constexpr int want = (RZ * GZ * GY > RY * GY * GZ ? RZ * GZ * GY : RY * GY * GZ);
    constexpr int r32 = want < 32 ? 32 : (want + 31) / 32 * 32;
    return RY == 16 && RZ == 16 ? (r32 < yz_threads<T>() ? r32 : yz_threads<T>()) : r32;
}
template <typename T, int RY, int GY, int RZ, int GZ>
__host__ __device__ constexpr int yz_bound() { return RY == 16 && RZ == 16 ? yz_threads<T>() : yz_nt<T, RY, GY, RZ, GZ>(); }

// ---- x forward ---------------------------------------------------------------------------------------------
// Each warp works alone on its 32 / GX rows: the split step writes X_k of its rows straight to the plane layout
// spec[k][row] (the rows of a warp are consecutive, so each frequency is one contiguous 32-byte or longer piece).
template <typename T, int RX, int GX>
__global__ void __launch_bounds__(x_threads<T>()) k_reg_x_fwd(PoissonArgs<T> A)
{
    pdl_enter();
    using C = typename CxT<T>::type;
    using SX = RegShape<RX, GX>;
    constexpr int M = RX * GX, NT = x_threads<T>(), B = NT / GX, P = 32 / GX, Q = SX::Q;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int SPX = A.reg_spx;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* twr = tw + M;
    C* rowbuf = twr + (M + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = group_of<GX>(lane), t = member_of<GX>(lane);
    const int b = warp * P + gi;
    const int rows = A.ny * A.nz, row = blockIdx.x * B + b;
    const bool act = row < rows;
    C v[SX::V];
    {   // the row's loads are issued before the tables are staged
        const T* __restrict__ src = A.f + (long long)(act ? row : 0) * A.nx;
#pragma unroll
        for (int m = 0; m < RX; ++m)
            v[m] = act ? *reinterpret_cast<const C*>(src + 2 * (t + GX * m)) : mk<C>(T(0), T(0));
    }
    stage_table(tw, A.twx, M);
    stage_table(twr, A.twr, M + 1);
    __syncthreads();
    C* rb = rowbuf + b * SPX;
    auto buf = [rb](int e) -> C& { return rb[e]; };
    reg_fwd<C, RX, GX>(v, t, tw, buf);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int k2 = 0; k2 < GX; ++k2)
            if (SX::valid(t, q)) rb[SX::slot(t, q, k2)] = v[q * GX + k2];
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
    // k = t + GX i for i = 0..RX/2 (k = M / 2 only for t = 0)
#pragma unroll
    for (int i = 0; i <= RX / 2; ++i) {
        const int k = t + GX * i;
        if (k > M / 2) break;
        const C Zk = rb[slot_of_freq<RX, GX>(k)];
        if (k == 0) {
            put(0, mk<C>(Zk.x + Zk.y, Zk.x - Zk.y));                  // (X_0, X_{nx/2})
            continue;
        }
        const C Zm = rb[slot_of_freq<RX, GX>(M - k)];
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
template <typename T, int RX, int GX>
__global__ void __launch_bounds__(x_threads<T>()) k_reg_x_inv(PoissonArgs<T> A)
{
    pdl_enter();
    using C = typename CxT<T>::type;
    using SX = RegShape<RX, GX>;
    constexpr int M = RX * GX, NT = x_threads<T>(), B = NT / GX, P = 32 / GX, Q = SX::Q;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int SPX = A.reg_spx;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* twr = tw + M;
    C* rowbuf = twr + (M + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gi = group_of<GX>(lane), t = member_of<GX>(lane);
    const int b = warp * P + gi;
    const int rows = A.ny * A.nz, row = blockIdx.x * B + b;
    const bool act = row < rows;
    // the pairs (X_k, X_{M-k}) of this thread, k = t + GX i: straight from the plane layout with all loads in
    // flight together (the twiddle tables are staged after them, so that their latencies overlap), or (rows of 256
    // frequencies) gathered first for the CTA's B rows into a frequency-major stage
    constexpr bool STAGED = GX == 16;
    constexpr int SB = B + 1;
    C* stage = rowbuf + B * SPX;
    C xk[RX / 2 + 1], xm[RX / 2 + 1];
    if (STAGED) {
        stage_table(tw, A.twx, M);
        stage_table(twr, A.twr, M + 1);
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
        for (int i = 0; i <= RX / 2; ++i) {
            const int k = t + GX * i;
            const bool ok = k <= M / 2;
            xk[i] = ok ? stage[k * SB + b] : mk<C>(T(0), T(0));
            xm[i] = ok && k > 0 ? stage[(M - k) * SB + b] : mk<C>(T(0), T(0));
        }
    } else {
        const C* __restrict__ spec = reinterpret_cast<const C*>(A.spec) + (act ? row : 0);
#pragma unroll
        for (int i = 0; i <= RX / 2; ++i) {
            const int k = t + GX * i;
            const bool ok = act && k <= M / 2;
            xk[i] = ok ? spec[(long long)k * rows] : mk<C>(T(0), T(0));
            xm[i] = ok && k > 0 ? spec[(long long)(M - k) * rows] : mk<C>(T(0), T(0));
        }
        stage_table(tw, A.twx, M);
        stage_table(twr, A.twr, M + 1);
        __syncthreads();   // tables staged
    }
    C* rb = rowbuf + b * SPX;
    // join: Z'_k = (X_k + conj X_{M-k}) + i W^{-k} (X_k - conj X_{M-k})
#pragma unroll
    for (int i = 0; i <= RX / 2; ++i) {
        const int k = t + GX * i;
        if (k > M / 2) break;
        const C Xk = xk[i], Xm = xm[i];
        if (k == 0) {
            rb[slot_of_freq<RX, GX>(0)] = mk<C>(Xk.x + Xk.y, Xk.x - Xk.y);
            continue;
        }
        {
            const C s = mk<C>(Xk.x + Xm.x, Xk.y - Xm.y), d = mk<C>(Xk.x - Xm.x, Xk.y + Xm.y);
            C w = twr[k];
            w.y = -w.y;
            const C wd = cmul(w, d);
            rb[slot_of_freq<RX, GX>(k)] = mk<C>(s.x - wd.y, s.y + wd.x);
        }
        if (2 * k != M) {
            const C s = mk<C>(Xm.x + Xk.x, Xm.y - Xk.y), d = mk<C>(Xm.x - Xk.x, Xm.y + Xk.y);
            C w = twr[M - k];
            w.y = -w.y;
            const C wd = cmul(w, d);
            rb[slot_of_freq<RX, GX>(M - k)] = mk<C>(s.x - wd.y, s.y + wd.x);
        }
    }
    __syncwarp();
    C v[SX::V];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int k2 = 0; k2 < GX; ++k2)
            v[q * GX + k2] = SX::valid(t, q) ? rb[SX::slot(t, q, k2)] : mk<C>(T(0), T(0));
    auto buf = [rb](int e) -> C& { return rb[e]; };
    reg_inv<C, RX, GX>(v, t, tw, buf);
    if (act) {
        T* __restrict__ dst = A.p + (long long)row * A.nx;
#pragma unroll
        for (int m = 0; m < RX; ++m) *reinterpret_cast<C*>(dst + 2 * (t + GX * m)) = v[m];
    }
}

// ---- (y, z) plane of one kx ----------------------------------------------------------------------------------
template <typename T, int RY, int GY, int RZ, int GZ>
__global__ void __launch_bounds__((yz_bound<T, RY, GY, RZ, GZ>())) k_reg_yz_solve(PoissonArgs<T> A)
{
    pdl_enter();
    using C = typename CxT<T>::type;
    using SY = RegShape<RY, GY>;
    using SZ = RegShape<RZ, GZ>;
    constexpr int NY = RY * GY, NZ = RZ * GZ, QY = SY::Q, QZ = SZ::Q;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int SP = A.reg_sp;
    // row z at z * SP, slot s of the y transform at s; row NZ and column NY (SP > NY when a warp's last z groups
    // run past NY) are the exchange slices of the groups past the last row or column, which hold no data
    C* plane = reinterpret_cast<C*>(smem_raw);
    C* twy = plane + (NZ + 1) * SP;
    C* twz = twy + NY;
    const int kx = blockIdx.x;
    C* g = reinterpret_cast<C*>(A.spec) + (long long)kx * NY * NZ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    // y forward: a group per z row, global memory -> registers -> shared plane (slots); the first row's loads are
    // issued before the twiddle tables are staged, so that their latencies overlap
    {
        constexpr int P = 32 / GY;
        const int gi = group_of<GY>(lane), t = member_of<GY>(lane);
        C v[SY::V];
        auto load_row = [&](int z) {
#pragma unroll
            for (int m = 0; m < RY; ++m) v[m] = z < NZ ? g[z * NY + t + GY * m] : mk<C>(T(0), T(0));
        };
        load_row(warp * P + gi);
        stage_table(twy, A.twy, NY);
        stage_table(twz, A.twz, NZ);
        __syncthreads();
        for (int z0 = warp * P; z0 < NZ; z0 += nwarps * P) {
            const int z = z0 + gi;
            const bool act = z < NZ;
            if (z0 != warp * P) load_row(z);
            C* row = plane + (act ? z : NZ) * SP;
            auto buf = [row](int e) -> C& { return row[e]; };
            reg_fwd<C, RY, GY>(v, t, twy, buf);
            __syncwarp();
            if (act) {
#pragma unroll
                for (int q = 0; q < QY; ++q)
#pragma unroll
                    for (int k2 = 0; k2 < GY; ++k2)
                        if (SY::valid(t, q)) row[SY::slot(t, q, k2)] = v[q * GY + k2];
            }
        }
    }
    __syncthreads();
    // z: a group per column (y slot c): forward FFT, x 1 / (lambda N), inverse FFT, in place in the column
    {
        constexpr int P = 32 / GZ;
        const int gi = group_of<GZ>(lane), t = member_of<GZ>(lane);
        const T lx = __ldg(A.lamx + kx);
        for (int c0 = warp * P; c0 < NY; c0 += nwarps * P) {
            const int c = c0 + gi;
            const bool act = c < NY;
            const int cc = act ? c : NY;
            const int ky = freq_of_slot<RY, GY>(act ? c : 0);
            const T lxy = lx + __ldg(A.lamy + ky);
            const bool ky_null = (kx == 0) && (ky == 0 || 2 * ky == NY);
            C v[SZ::V];
#pragma unroll
            for (int m = 0; m < RZ; ++m) v[m] = plane[(t + GZ * m) * SP + cc];
            auto buf = [plane, SP, cc](int e) -> C& { return plane[e * SP + cc]; };
            reg_fwd<C, RZ, GZ>(v, t, twz, buf);
#pragma unroll
            for (int q = 0; q < QZ; ++q)
#pragma unroll
                for (int k2 = 0; k2 < GZ; ++k2) {
                    if (!SZ::valid(t, q)) continue;   // a transform past R: nothing to scale
                    const int kz = SZ::freq(t, q, k2);
                    const bool null = ky_null && (kz == 0 || 2 * kz == NZ);
                    const T s = null ? T(0) : inv_lambda(A.invN, lxy + __ldg(A.lamz + kz));
                    v[q * GZ + k2] = cscale(v[q * GZ + k2], s);
                }
            reg_inv<C, RZ, GZ>(v, t, twz, buf);
            __syncwarp();
            if (act) {
#pragma unroll
                for (int m = 0; m < RZ; ++m) plane[(t + GZ * m) * SP + cc] = v[m];
            }
        }
    }
    __syncthreads();
    // y inverse: a group per z row, shared plane -> registers -> global memory
    {
        constexpr int P = 32 / GY;
        const int gi = group_of<GY>(lane), t = member_of<GY>(lane);
        for (int z0 = warp * P; z0 < NZ; z0 += nwarps * P) {
            const int z = z0 + gi;
            const bool act = z < NZ;
            C* row = plane + (act ? z : NZ) * SP;
            C v[SY::V];
#pragma unroll
            for (int q = 0; q < QY; ++q)
#pragma unroll
                for (int k2 = 0; k2 < GY; ++k2)
                    v[q * GY + k2] = SY::valid(t, q) ? row[SY::slot(t, q, k2)] : mk<C>(T(0), T(0));
            auto buf = [row](int e) -> C& { return row[e]; };
            reg_inv<C, RY, GY>(v, t, twy, buf);
            if (act) {
#pragma unroll
                for (int m = 0; m < RY; ++m) g[z * NY + t + GY * m] = v[m];
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
        reg_fwd<C, 16, GY>(v, t, tw, buf);
        if (act) {
#pragma unroll
            for (int q = 0; q < Q; ++q)
#pragma unroll
                for (int k2 = 0; k2 < GY; ++k2) g[RegShape<16, GY>::slot(t, q, k2)] = v[q * GY + k2];
        }
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int k2 = 0; k2 < GY; ++k2)
                v[q * GY + k2] = act ? g[RegShape<16, GY>::slot(t, q, k2)] : mk<C>(T(0), T(0));
        reg_inv<C, 16, GY>(v, t, tw, buf);
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
    reg_fwd<C, 16, GZ>(v, t, twz, buf);
#pragma unroll
    for (int q = 0; q < QZ; ++q)
#pragma unroll
        for (int k2 = 0; k2 < GZ; ++k2) {
            const int kz = RegShape<16, GZ>::freq(t, q, k2);
            const bool null = ky_null && (kz == 0 || 2 * kz == NZ);
            const T s = null ? T(0) : inv_lambda(A.invN, lxy + __ldg(A.lamz + kz));
            v[q * GZ + k2] = cscale(v[q * GZ + k2], s);
        }
    reg_inv<C, 16, GZ>(v, t, twz, buf);
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
// Register transform shape of an axis of n points: R values per thread and G threads, n = R G.  Lengths 16 G
// (G = 1..16) in both precisions; the 2-3-5 lengths of the batch and serving rooms (36 .. 96) in FP32, whose
// (y, z) planes fit whole in shared memory.  Some take more threads than divide R (9 x 4, 15 x 4, 9 x 8 and, along
// x, 5 x 8, 6 x 8, 10 x 8, 12 x 8): short first-stage DFTs and four or eight threads per transform instead of up
// to 36 values on two threads (the 72 x 72 plane kernel: 12.3 us instead of 16.4 with 36 x 2).  The x passes
// prefer eight threads (32 points: 6.5 instead of 8.3 us per pass as 4 x 8, 64: 6.8 instead of 8.0 as 8 x 8, 96:
// 9.2 instead of 10.3 as 12 x 8; 128 stays 16 x 8: 14 against 12.5 us as 8 x 16); the plane kernel prefers the
// 4-thread groups of adjacent lanes (80 x 80 as 20 x 4: 12.6 us, as 10 x 8: 14.6).
bool reg_shape(int n, bool fp32, int* R, int* G, bool x_axis = false)
{
    if (fp32 && x_axis && (n == 32 || n == 64)) { *R = n / 8; *G = 8; return true; }
    for (int g = 1; g <= 16; g *= 2)
        if (n == 16 * g) { *R = 16; *G = g; return true; }
    if (!fp32) return false;
    static const int tab_yz[][3] = {{36, 9, 4}, {40, 20, 2}, {48, 12, 4}, {60, 15, 4}, {72, 9, 8}, {80, 20, 4},
                                    {96, 24, 4}};
    static const int tab_x[][3] = {{36, 9, 4}, {40, 5, 8}, {48, 6, 8}, {60, 15, 4}, {72, 9, 8}, {80, 10, 8},
                                   {96, 12, 8}};
    for (const auto& e : x_axis ? tab_x : tab_yz)
        if (n == e[0]) { *R = e[1]; *G = e[2]; return true; }
    return false;
}

// Shared-memory wavefronts of a warp access, worst over its steps: the warp's lanes are served in 128-byte phases
// (all 32 lanes for 4-byte elements, half-warps for 8-byte, quarter-warps for 16-byte), a phase taking as many
// wavefronts as the most distinct 4-byte words any of its 32 banks holds.  addr(lane, step) in elements of esz
// bytes, for steps 0..nsteps-1; the ideal is 32 esz / 128 wavefronts.
template <typename F>
int worst_ways(int esz, int nsteps, F addr)
{
    const int per_phase = esz > 4 ? 128 / esz : 32;
    int worst = 1;
    for (int step = 0; step < nsteps; ++step) {
        int total = 0;
        for (int p0 = 0; p0 < 32; p0 += per_phase) {
            int ways[32] = {0};
            long long seen[32][32];
            int nseen[32] = {0};
            for (int lane = p0; lane < p0 + per_phase; ++lane) {
                const long long e = addr(lane, step);
                if (e < 0) continue;   // this lane makes no access at this step
                const long long byte = e * (long long)esz;
                for (int w = 0; w < esz / 4; ++w) {
                    const long long word = byte / 4 + w;
                    const int bank = (int)(word % 32);
                    bool dup = false;
                    for (int i = 0; i < nseen[bank]; ++i) dup |= seen[bank][i] == word;
                    if (!dup && nseen[bank] < 32) { seen[bank][nseen[bank]++] = word; ways[bank]++; }
                }
            }
            int m = 1;
            for (int i = 0; i < 32; ++i) m = ways[i] > m ? ways[i] : m;
            total += m;
        }
        worst = total > worst ? total : worst;
    }
    return worst;
}

int q_h(int R, int G) { return (R + G - 1) / G; }
int xpos_h(int R, int G, int t, int k1) { const int Q = q_h(R, G); return k1 * G + ((t + k1 / Q) & (G - 1)); }
// slot of held value (q, k2) of thread t, -1 past R (RegShape::slot)
long long slot_h(int R, int G, int t, int q, int k2)
{
    const int Q = q_h(R, G);
    if (t * Q + q >= R) return -1;
    return R % G == 0 ? t + G * q + (long long)R * k2 : t * Q + q + (long long)R * k2;
}

// group and member of a lane (adjacent: a group's threads are adjacent lanes, the plane and x kernels for G = 4;
// else member i of group g is lane g + i 32 / G)
struct LaneMap {
    int G;
    bool adj;
    int grp(int l) const { return adj ? l / G : l % (32 / G); }
    int mem(int l) const { return adj ? l % G : l / (32 / G); }
};

// wavefronts of the row-owned accesses (a group of G threads per row, rows `stride` apart)
int row_ways(int R, int G, int stride, int esz, bool adj)
{
    const int Q = q_h(R, G);
    const LaneMap L{G, adj};
    int w = 0;
    auto mx = [&](int v) { w = v > w ? v : w; };
    if (G > 1) {
        // exchange: the R first-stage outputs written, then per held transform q the G sources read
        mx(worst_ways(esz, R, [&](int l, int s) { return (long long)L.grp(l) * stride + xpos_h(R, G, L.mem(l), s); }));
        mx(worst_ways(esz, Q * G, [&](int l, int s) {
            const int k1 = L.mem(l) * Q + s / G;
            return k1 < R ? (long long)L.grp(l) * stride + xpos_h(R, G, s % G, k1) : -1LL; }));
    }
    mx(worst_ways(esz, Q * G, [&](int l, int s) {   // held values to and from their slots
        const long long e = slot_h(R, G, L.mem(l), s % Q, s / Q);
        return e < 0 ? -1LL : (long long)L.grp(l) * stride + e; }));
    return w;
}

// wavefronts of the column-owned accesses (element e of column c at e * stride + c)
int col_ways(int R, int G, int stride, int esz, bool adj)
{
    const int Q = q_h(R, G);
    const LaneMap L{G, adj};
    int w = 0;
    auto mx = [&](int v) { w = v > w ? v : w; };
    mx(worst_ways(esz, R, [&](int l, int s) { return (long long)(L.mem(l) + G * s) * stride + L.grp(l); }));
    if (G > 1) {
        mx(worst_ways(esz, R, [&](int l, int s) { return (long long)xpos_h(R, G, L.mem(l), s) * stride + L.grp(l); }));
        mx(worst_ways(esz, Q * G, [&](int l, int s) {
            const int k1 = L.mem(l) * Q + s / G;
            return k1 < R ? (long long)xpos_h(R, G, s % G, k1) * stride + L.grp(l) : -1LL; }));
    }
    return w;
}

template <typename T>
size_t x_smem(int M, int G, int spx)
{
    const int B = x_threads<T>() / G;
    const size_t stage = G == 16 ? (size_t)M * (B + 1) : 0;     // the frequency-major stage of 256-point rows
    return ((size_t)M + (M + 1) + (size_t)B * spx + stage) * sizeof(typename CxT<T>::type);
}

template <typename T>
size_t yz_smem(int ny, int nz, int sp)
{
    return ((size_t)(nz + 1) * sp + ny + nz) * sizeof(typename CxT<T>::type);
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

// ---- tile mode (lengths 16 G) --------------------------------------------------------------------------------
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

// ---- shape dispatch ------------------------------------------------------------------------------------------
// Calls f.template run<R, G>() for the shape (r, g) of set SET: kShapes16 the lengths 16 G (both precisions),
// kShapesYZ adds the FP32 2-3-5 shapes of the y and z axes, kShapesX those of the x axis (no double or unused
// instantiations of them).
constexpr int kShapes16 = 0, kShapesYZ = 1, kShapesX = 2;

template <typename T, int SET, typename F>
cudaError_t with_shape(int r, int g, F&& f)
{
    if (r == 16) {
        switch (g) {
            case 1: return f.template run<16, 1>();
            case 2: return f.template run<16, 2>();
            case 4: return f.template run<16, 4>();
            case 8: return f.template run<16, 8>();
            case 16: return f.template run<16, 16>();
            default: return cudaErrorInvalidValue;
        }
    }
    if constexpr (sizeof(T) == 4 && SET != kShapes16) {
        if (r == 9 && g == 4) return f.template run<9, 4>();
        if (r == 15 && g == 4) return f.template run<15, 4>();
        if (r == 9 && g == 8) return f.template run<9, 8>();
        if constexpr (SET == kShapesYZ) {
            if (r == 20 && g == 2) return f.template run<20, 2>();
            if (r == 12 && g == 4) return f.template run<12, 4>();
            if (r == 20 && g == 4) return f.template run<20, 4>();
            if (r == 24 && g == 4) return f.template run<24, 4>();
        } else {
            if (r == 5 && g == 8) return f.template run<5, 8>();
            if (r == 6 && g == 8) return f.template run<6, 8>();
            if (r == 8 && g == 8) return f.template run<8, 8>();
            if (r == 10 && g == 8) return f.template run<10, 8>();
            if (r == 12 && g == 8) return f.template run<12, 8>();
            if (r == 4 && g == 8) return f.template run<4, 8>();
        }
    }
    return cudaErrorInvalidValue;
}

template <typename T>
struct XLaunch {
    const PoissonArgs<T>& a;
    bool fwd;
    cudaStream_t st;
    bool prepare;
    template <int R, int G>
    cudaError_t run() const
    {
        constexpr int B = x_threads<T>() / G;
        const size_t sm = x_smem<T>(R * G, G, a.reg_spx);
        if (prepare) {
            cudaError_t e = raise_smem(k_reg_x_fwd<T, R, G>, sm);
            return e == cudaSuccess ? raise_smem(k_reg_x_inv<T, R, G>, sm) : e;
        }
        const int rows = a.ny * a.nz;
        const unsigned grid = (unsigned)((rows + B - 1) / B);
        return launch_pdl(fwd ? k_reg_x_fwd<T, R, G> : k_reg_x_inv<T, R, G>, dim3(grid), dim3(x_threads<T>()), sm,
                          st, a);
    }
};

template <typename T>
cudaError_t dispatch_x(const PoissonArgs<T>& a, bool fwd, cudaStream_t st, bool prepare = false)
{
    return with_shape<T, kShapesX>(a.rx, a.gx, XLaunch<T>{a, fwd, st, prepare});
}

template <typename T, int RY, int GY>
struct YZLaunch {
    const PoissonArgs<T>& a;
    cudaStream_t st;
    bool prepare;
    template <int RZ, int GZ>
    cudaError_t run() const
    {
        const size_t sm = yz_smem<T>(a.ny, a.nz, a.reg_sp);
        if (prepare) return raise_smem(k_reg_yz_solve<T, RY, GY, RZ, GZ>, sm);
        return launch_pdl(k_reg_yz_solve<T, RY, GY, RZ, GZ>, dim3(a.M), dim3(yz_nt<T, RY, GY, RZ, GZ>()), sm, st,
                          a);
    }
};

template <typename T>
struct YLaunch {
    const PoissonArgs<T>& a;
    cudaStream_t st;
    bool prepare;
    template <int RY, int GY>
    cudaError_t run() const
    {
        if (RY != 16 && (a.rz != RY || a.gz != GY)) return cudaErrorInvalidValue;   // 2-3-5 planes: ny == nz
        if constexpr (RY != 16) {
            return YZLaunch<T, RY, GY>{a, st, prepare}.template run<RY, GY>();
        } else {
            if (a.rz != 16) return cudaErrorInvalidValue;
            return with_shape<T, kShapes16>(16, a.gz, YZLaunch<T, RY, GY>{a, st, prepare});
        }
    }
};

template <typename T>
cudaError_t dispatch_yz(const PoissonArgs<T>& a, cudaStream_t st, bool prepare = false)
{
    return with_shape<T, kShapesYZ>(a.ry, a.gy, YLaunch<T>{a, st, prepare});
}

}  // namespace

template <typename T>
bool RegFft<T>::eligible(int nx, int ny, int nz)
{
    if (nx % 2) return false;
    constexpr bool fp32 = sizeof(T) == 4;
    int rx, gx, ry, gy, rz, gz;
    if (!reg_shape(nx / 2, fp32, &rx, &gx, true) || !reg_shape(ny, fp32, &ry, &gy) || !reg_shape(nz, fp32, &rz, &gz))
        return false;
    if (x_smem<T>(nx / 2, gx, nx / 2 + 15) > kRegSmemLimit) return false;
    // 2-3-5 lengths in y or z: square planes that fit whole (no tile mode); 16 G lengths: tiles when they do not
    if (ry != 16 || rz != 16)
        return ry == rz && gy == gz && yz_smem<T>(ny, nz, ny + 15) <= kRegSmemLimit;
    return y_smem<T>(ny, ny + 15) <= kRegSmemLimit;
}

template <typename T>
void RegFft<T>::configure(PoissonArgs<T>& a)
{
    a.reg = 0;
    if (!eligible(a.nx, a.ny, a.nz)) return;
    constexpr bool fp32 = sizeof(T) == 4;
    reg_shape(a.M, fp32, &a.rx, &a.gx, true);
    reg_shape(a.ny, fp32, &a.ry, &a.gy);
    reg_shape(a.nz, fp32, &a.rz, &a.gz);
    const int esz = (int)sizeof(typename CxT<T>::type);
    auto adj = [](int g) { return g == 4; };   // adjacent_groups<G>() of the plane and x kernels
    // plane stride: fewest bank conflicts over the y-row and z-column accesses, then the smallest
    // (a pad column holds the exchange of the z groups past the last y slot when a warp's groups run past ny)
    int best = -1, best_w = 1 << 30;
    for (int pad = a.ny % (32 / a.gz) ? 1 : 0; pad < 16; ++pad) {
        const int sp = a.ny + pad;
        const int w = std::max(row_ways(a.ry, a.gy, sp, esz, adj(a.gy)), col_ways(a.rz, a.gz, sp, esz, adj(a.gz)));
        if (w < best_w) { best_w = w; best = sp; }
    }
    a.reg_sp = best;
    const bool pow2 = a.ry == 16 && a.rz == 16;
    a.reg_tile = pow2 && (yz_smem<T>(a.ny, a.nz, a.reg_sp) > kRegSmemLimit || std::getenv("VF_REG_TILE")) ? 1 : 0;
    if (a.reg_tile) {
        // y passes: the row slices of the groups; z tile: TB slots of one plane, columns as for the plane
        best = -1; best_w = 1 << 30;
        for (int pad = 0; pad < 16; ++pad) {
            const int w = row_ways(16, a.gy, a.ny + pad, esz, false);
            if (w < best_w) { best_w = w; best = a.ny + pad; }
        }
        a.reg_sy = best;
        a.reg_tb = std::min(a.ny, 256 / a.gz);
        best = -1; best_w = 1 << 30;
        for (int pad = 0; pad < 16; ++pad) {
            const int w = col_ways(16, a.gz, a.reg_tb + pad, esz, false);
            if (w < best_w) { best_w = w; best = a.reg_tb + pad; }
        }
        a.reg_st = best;
    }
    // x passes: the row slices of the groups
    best = -1; best_w = 1 << 30;
    for (int pad = 0; pad < 16; ++pad) {
        const int w = row_ways(a.rx, a.gx, a.M + pad, esz, adj(a.gx));
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
    cudaError_t e = dispatch_x<T>(a, true, nullptr, true);
    if (e != cudaSuccess) return e;
    if (a.reg_tile) {
        if ((e = prepare_tile<T, 1>(a)) != cudaSuccess) return e;
        if ((e = prepare_tile<T, 2>(a)) != cudaSuccess) return e;
        if ((e = prepare_tile<T, 4>(a)) != cudaSuccess) return e;
        if ((e = prepare_tile<T, 8>(a)) != cudaSuccess) return e;
        return prepare_tile<T, 16>(a);
    }
    return dispatch_yz<T>(a, nullptr, true);
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
