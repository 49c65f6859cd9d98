// FFT Poisson solve of the pressure equation (Sec. 2.2, Eq. 9): p^{k+1} = L^{-1}[ D u* + D((1 - beta) G p^k) ].
//
// One iteration is five passes over a half spectrum that stays resident in L2 for rooms up to ~10^7 cells:
//   x forward  : builds the right-hand side f from r, p^k and the mask, real-to-complex FFT along x
//                (two real points packed per complex value, nx/2-point complex FFT, then the split step);
//   y forward  : complex FFT along y;
//   z solve    : complex FFT along z, multiply by 1 / (lambda N) (0 on the null modes), inverse FFT along z;
//   y inverse  : complex inverse FFT along y;
//   x inverse  : complex-to-real inverse FFT along x, writes p^{k+1}.
// The spectrum has nx/2 complex columns per (y, z) row.  Column 0 holds the x-spectra at kx = 0 (real part)
// and kx = nx/2 (imaginary part): both are real for real data and both have sin^2(2 pi kx / nx) = 0, so the
// y/z transforms and the eigenvalue division treat the packed pair exactly like any other column.
//
// Each CTA runs a mixed-radix (2, 3, 4, 5, 8) Stockham FFT in shared memory over a batch of sequences: rows of
// the x passes (one row per sequence), or a tile of consecutive kx columns for the y and z passes (so every global
// access is a contiguous run of cols_per_block complex values).
#include <cuda_runtime.h>

#include <cstdint>

#include "vf_internal.h"

namespace vf {
namespace {

template <typename T> struct CxT;
template <> struct CxT<float> { using type = float2; };
template <> struct CxT<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) { C r; r.x = a; r.y = b; return r; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
// multiply by +i (INV) or -i (forward): the rotation of a forward / inverse DFT of order 4
template <typename C, bool INV> __device__ __forceinline__ C rot(C a) { return INV ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x); }

// ---- small DFTs in registers: X_k = sum_m v_m exp(-+ 2 pi i m k / R) (minus forward, plus inverse) ----------
template <typename C, bool INV>
__device__ __forceinline__ void dft2(C& a, C& b) { const C t = a; a = cadd(t, b); b = csub(t, b); }

template <typename C, bool INV>
__device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3)
{
    const C t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3), t3 = rot<C, INV>(csub(v1, v3));
    v0 = cadd(t0, t2); v2 = csub(t0, t2); v1 = cadd(t1, t3); v3 = csub(t1, t3);
}

template <typename C, bool INV>
__device__ __forceinline__ void dft3(C& v0, C& v1, C& v2)
{
    using R = decltype(C::x);
    const R s3 = R(0.86602540378443864676);   // sin(2 pi / 3)
    const C t = cadd(v1, v2);
    const C m = mk<C>(v0.x - R(0.5) * t.x, v0.y - R(0.5) * t.y);
    const C d = rot<C, INV>(cscale(csub(v1, v2), s3));
    v0 = cadd(v0, t); v1 = cadd(m, d); v2 = csub(m, d);
}

template <typename C, bool INV>
__device__ __forceinline__ void dft5(C& v0, C& v1, C& v2, C& v3, C& v4)
{
    using R = decltype(C::x);
    const R c1 = R(0.30901699437494742410), c2 = R(-0.80901699437494742410);   // cos(2 pi/5), cos(4 pi/5)
    const R s1 = R(0.95105651629515357212), s2 = R(0.58778525229247312917);    // sin(2 pi/5), sin(4 pi/5)
    const C t1 = cadd(v1, v4), t2 = cadd(v2, v3), d1 = csub(v1, v4), d2 = csub(v2, v3);
    const C a1 = mk<C>(v0.x + c1 * t1.x + c2 * t2.x, v0.y + c1 * t1.y + c2 * t2.y);
    const C a2 = mk<C>(v0.x + c2 * t1.x + c1 * t2.x, v0.y + c2 * t1.y + c1 * t2.y);
    const C b1 = rot<C, INV>(mk<C>(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
    const C b2 = rot<C, INV>(mk<C>(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
    v0 = cadd(v0, cadd(t1, t2));
    v1 = cadd(a1, b1); v4 = csub(a1, b1);
    v2 = cadd(a2, b2); v3 = csub(a2, b2);
}

template <typename C, bool INV>
__device__ __forceinline__ void dft8(C* v)
{
    using R = decltype(C::x);
    const R h = R(0.70710678118654752440);
    dft4<C, INV>(v[0], v[2], v[4], v[6]);
    dft4<C, INV>(v[1], v[3], v[5], v[7]);
    // odd outputs times W8^k, W8 = exp(-+ 2 pi i / 8)
    const C o1 = INV ? mk<C>(h * (v[3].x - v[3].y), h * (v[3].x + v[3].y))
                     : mk<C>(h * (v[3].x + v[3].y), h * (v[3].y - v[3].x));
    const C o2 = rot<C, INV>(v[5]);
    const C o3 = INV ? mk<C>(-h * (v[7].x + v[7].y), h * (v[7].x - v[7].y))
                     : mk<C>(h * (v[7].y - v[7].x), -h * (v[7].x + v[7].y));
    const C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <typename C, int R, bool INV>
__device__ __forceinline__ void dft(C* v)
{
    if (R == 2) dft2<C, INV>(v[0], v[1]);
    else if (R == 3) dft3<C, INV>(v[0], v[1], v[2]);
    else if (R == 4) dft4<C, INV>(v[0], v[1], v[2], v[3]);
    else if (R == 5) dft5<C, INV>(v[0], v[1], v[2], v[3], v[4]);
    else dft8<C, INV>(v);
}

// One radix-R Stockham pass over nseq sequences of length n held in shared memory: element k of sequence b
// lives at k * es + b * ss.  Ns is the product of the radices already applied.  Work item (j, b) reads
// src[j + r n/R], twiddles by W_n^(r (j mod Ns) n / (Ns R)), does a DFT of order R and writes
// dst[(j / Ns) Ns R + (j mod Ns) + r Ns].  tw[m] = exp(-2 pi i m / n).
template <typename C, int R, bool INV, bool SEQFAST>
__device__ __forceinline__ void stockham_pass(const C* __restrict__ src, C* __restrict__ dst, int n, int nseq,
                                              int es, int ss, int Ns, const C* __restrict__ tw)
{
    const int nb = n / R;
    const int total = nb * nseq;
    const int tstride = n / (Ns * R);
    for (int it = threadIdx.x; it < total; it += blockDim.x) {
        int j, b;
        if (SEQFAST) { b = it % nseq; j = it / nseq; }
        else { j = it % nb; b = it / nb; }
        const int jm = j % Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[(j + r * nb) * es + b * ss];
        if (jm) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = tw[jm * r * tstride];
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft<C, R, INV>(v);
        const int d0 = (j - jm) * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(d0 + r * Ns) * es + b * ss] = v[r];
    }
}

// Full FFT of every sequence; buffers a (input) and b (scratch) alternate; returns the one holding the result.
template <typename C, bool INV, bool SEQFAST>
__device__ C* fft_block(C* a, C* b, const FftAxis& ax, int nseq, int es, int ss, const C* tw)
{
    int Ns = 1;
    for (int s = 0; s < ax.nstages; ++s) {
        const int R = ax.radix[s];
        switch (R) {
            case 2: stockham_pass<C, 2, INV, SEQFAST>(a, b, ax.n, nseq, es, ss, Ns, tw); break;
            case 3: stockham_pass<C, 3, INV, SEQFAST>(a, b, ax.n, nseq, es, ss, Ns, tw); break;
            case 4: stockham_pass<C, 4, INV, SEQFAST>(a, b, ax.n, nseq, es, ss, Ns, tw); break;
            case 5: stockham_pass<C, 5, INV, SEQFAST>(a, b, ax.n, nseq, es, ss, Ns, tw); break;
            default: stockham_pass<C, 8, INV, SEQFAST>(a, b, ax.n, nseq, es, ss, Ns, tw); break;
        }
        __syncthreads();
        C* t = a; a = b; b = t;
        Ns *= R;
    }
    return a;
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Right-hand side of Eq. 9 at one cell: f = r + sum_j (1/(2h_j))^2 [(1 - beta^+)(p^{++} - p^0) - (1 - beta^-)(p^0 - p^{--})]
// (= r + sum_j delta_j((1 - beta) delta_j p) with central differences).
template <typename T>
__device__ __forceinline__ T poisson_rhs(const PoissonArgs<T>& A, int x, int y, int z)
{
    const long long nx = A.nx, ny = A.ny;
    const long long plane = nx * ny;
    const long long i = x + nx * (y + ny * (long long)z);
    T f = __ldg(A.r + i);
    if (!A.use_mask) return f;
    const int xm = wrapi(x - 1, A.nx), xp = wrapi(x + 1, A.nx);
    const int ym = wrapi(y - 1, A.ny), yp = wrapi(y + 1, A.ny);
    const int zm = wrapi(z - 1, A.nz), zp = wrapi(z + 1, A.nz);
    const long long zb = (long long)z * plane, yb = (long long)y * nx;
    const uint8_t bxm = __ldg(A.mask + zb + yb + xm) & kBitBeta, bxp = __ldg(A.mask + zb + yb + xp) & kBitBeta;
    const uint8_t bym = __ldg(A.mask + zb + ym * nx + x) & kBitBeta, byp = __ldg(A.mask + zb + yp * nx + x) & kBitBeta;
    const uint8_t bzm = __ldg(A.mask + zm * plane + yb + x) & kBitBeta, bzp = __ldg(A.mask + zp * plane + yb + x) & kBitBeta;
    if (bxm & bxp & bym & byp & bzm & bzp) return f;   // all six neighbours fluid: the correction vanishes
    const T p0 = __ldg(A.p + i);
    T corr = T(0);
    {
        const T pp = __ldg(A.p + zb + yb + wrapi(x + 2, A.nx)), pm = __ldg(A.p + zb + yb + wrapi(x - 2, A.nx));
        corr += A.i2h2[0] * ((bxp ? T(0) : (pp - p0)) - (bxm ? T(0) : (p0 - pm)));
    }
    {
        const T pp = __ldg(A.p + zb + wrapi(y + 2, A.ny) * nx + x), pm = __ldg(A.p + zb + wrapi(y - 2, A.ny) * nx + x);
        corr += A.i2h2[1] * ((byp ? T(0) : (pp - p0)) - (bym ? T(0) : (p0 - pm)));
    }
    {
        const T pp = __ldg(A.p + wrapi(z + 2, A.nz) * plane + yb + x), pm = __ldg(A.p + wrapi(z - 2, A.nz) * plane + yb + x);
        corr += A.i2h2[2] * ((bzp ? T(0) : (pp - p0)) - (bzm ? T(0) : (p0 - pm)));
    }
    return f + corr;
}

// ---- x forward: right-hand side + real-to-complex FFT along x ---------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_fft_x_fwd(PoissonArgs<T> A)
{
    using C = typename CxT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = A.M, nx = A.nx, B = A.rows_per_block;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + B * M;
    T* fr = reinterpret_cast<T*>(buf0);   // real view: row b, point x at fr[b * nx + x]
    const int rows = A.ny * A.nz;
    const int row0 = blockIdx.x * B;
    for (int it = threadIdx.x; it < B * nx; it += blockDim.x) {
        const int b = it / nx, x = it - b * nx, row = row0 + b;
        T v = T(0);
        if (row < rows) v = poisson_rhs(A, x, row % A.ny, row / A.ny);
        fr[it] = v;
    }
    __syncthreads();
    const C* tw = reinterpret_cast<const C*>(A.twx);
    const C* twr = reinterpret_cast<const C*>(A.twr);
    C* res = fft_block<C, false, false>(buf0, buf1, A.ax, B, 1, M, tw);
    C* spec = reinterpret_cast<C*>(A.spec);
    for (int it = threadIdx.x; it < B * M; it += blockDim.x) {
        const int b = it / M, k = it - b * M, row = row0 + b;
        if (row >= rows) continue;
        const C Zk = res[b * M + k];
        C X;
        if (k == 0) {
            X = mk<C>(Zk.x + Zk.y, Zk.x - Zk.y);                 // (X_0, X_{nx/2})
        } else {
            const C Zm = res[b * M + (M - k)];                  // conj taken below
            const C E = mk<C>(T(0.5) * (Zk.x + Zm.x), T(0.5) * (Zk.y - Zm.y));
            const C O = mk<C>(T(0.5) * (Zk.y + Zm.y), T(-0.5) * (Zk.x - Zm.x));
            X = cadd(E, cmul(__ldg(&twr[k]), O));               // X_k = E_k + W^k O_k
        }
        spec[(long long)row * M + k] = X;
    }
}

// ---- y pass (forward or inverse), in place on the spectrum --------------------------------------------------
template <typename T, bool INV>
__global__ void __launch_bounds__(256) k_fft_y(PoissonArgs<T> A)
{
    using C = typename CxT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TB = A.cols_per_block, n = A.ny, M = A.M;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + TB * n;
    const int kx0 = blockIdx.x * TB;
    const int z = blockIdx.y;
    C* spec = reinterpret_cast<C*>(A.spec);
    const long long base = (long long)z * n * M;
    for (int it = threadIdx.x; it < n * TB; it += blockDim.x) {
        const int y = it / TB, b = it - y * TB, kx = kx0 + b;
        buf0[it] = (kx < M) ? spec[base + (long long)y * M + kx] : mk<C>(T(0), T(0));
    }
    __syncthreads();
    C* res = fft_block<C, INV, true>(buf0, buf1, A.ay, TB, TB, 1, reinterpret_cast<const C*>(A.twy));
    for (int it = threadIdx.x; it < n * TB; it += blockDim.x) {
        const int y = it / TB, b = it - y * TB, kx = kx0 + b;
        if (kx < M) spec[base + (long long)y * M + kx] = res[it];
    }
}

// ---- z pass: forward FFT, division by the Laplacian eigenvalues, inverse FFT --------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_fft_z_solve(PoissonArgs<T> A)
{
    using C = typename CxT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TB = A.cols_per_block, n = A.nz, M = A.M, ny = A.ny;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + TB * n;
    const int kx0 = blockIdx.x * TB;
    const int ky = blockIdx.y;
    C* spec = reinterpret_cast<C*>(A.spec);
    const long long zstride = (long long)ny * M;
    const long long base = (long long)ky * M;
    for (int it = threadIdx.x; it < n * TB; it += blockDim.x) {
        const int z = it / TB, b = it - z * TB, kx = kx0 + b;
        buf0[it] = (kx < M) ? spec[base + z * zstride + kx] : mk<C>(T(0), T(0));
    }
    __syncthreads();
    const C* tw = reinterpret_cast<const C*>(A.twz);
    C* res = fft_block<C, false, true>(buf0, buf1, A.az, TB, TB, 1, tw);
    C* other = (res == buf0) ? buf1 : buf0;
    const T ly = __ldg(A.lamy + ky);
    const bool ky_null = (ky == 0) || (2 * ky == ny);
    for (int it = threadIdx.x; it < n * TB; it += blockDim.x) {
        const int kz = it / TB, b = it - kz * TB, kx = kx0 + b;
        T s = T(0);
        if (kx < M) {
            const bool null = (kx == 0) && ky_null && ((kz == 0) || (2 * kz == n));
            if (!null) s = A.invN / -(__ldg(A.lamx + kx) + ly + __ldg(A.lamz + kz));
        }
        res[it] = cscale(res[it], s);
    }
    __syncthreads();
    C* out = fft_block<C, true, true>(res, other, A.az, TB, TB, 1, tw);
    for (int it = threadIdx.x; it < n * TB; it += blockDim.x) {
        const int z = it / TB, b = it - z * TB, kx = kx0 + b;
        if (kx < M) spec[base + z * zstride + kx] = out[it];
    }
}

// ---- x inverse: complex-to-real FFT along x, writes p ---------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_fft_x_inv(PoissonArgs<T> A)
{
    using C = typename CxT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = A.M, nx = A.nx, B = A.rows_per_block;
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + B * M;
    const int rows = A.ny * A.nz;
    const int row0 = blockIdx.x * B;
    const C* spec = reinterpret_cast<const C*>(A.spec);
    for (int it = threadIdx.x; it < B * M; it += blockDim.x) {
        const int b = it / M, k = it - b * M, row = row0 + b;
        buf0[it] = (row < rows) ? spec[(long long)row * M + k] : mk<C>(T(0), T(0));
    }
    __syncthreads();
    const C* twr = reinterpret_cast<const C*>(A.twr);
    for (int it = threadIdx.x; it < B * M; it += blockDim.x) {
        const int b = it / M, k = it - b * M;
        const C Xk = buf0[it];
        C Z;
        if (k == 0) {
            Z = mk<C>(Xk.x + Xk.y, Xk.x - Xk.y);
        } else {
            const C Xm = buf0[b * M + (M - k)];                 // conj taken below
            const C s = mk<C>(Xk.x + Xm.x, Xk.y - Xm.y);        // X_k + conj(X_{M-k})
            const C d = mk<C>(Xk.x - Xm.x, Xk.y + Xm.y);        // X_k - conj(X_{M-k})
            C w = __ldg(&twr[k]);
            w.y = -w.y;                                         // W^{-k}
            const C wd = cmul(w, d);
            Z = mk<C>(s.x - wd.y, s.y + wd.x);                  // s + i W^{-k} d
        }
        buf1[it] = Z;
    }
    __syncthreads();
    C* res = fft_block<C, true, false>(buf1, buf0, A.ax, B, 1, M, reinterpret_cast<const C*>(A.twx));
    const T* fr = reinterpret_cast<const T*>(res);
    for (int it = threadIdx.x; it < B * nx; it += blockDim.x) {
        const int b = it / nx, x = it - b * nx, row = row0 + b;
        if (row < rows) A.p[(long long)row * nx + x] = fr[it];
    }
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

template <typename T>
size_t Kernels<T>::fft_smem_x(const PoissonArgs<T>& a)
{
    return 2 * (size_t)a.rows_per_block * a.M * sizeof(typename CxT<T>::type);
}

template <typename T>
size_t Kernels<T>::fft_smem_yz(const PoissonArgs<T>& a, int n)
{
    return 2 * (size_t)a.cols_per_block * n * sizeof(typename CxT<T>::type);
}

template <typename T>
cudaError_t Kernels<T>::poisson_prepare(const PoissonArgs<T>& a)
{
    const size_t sx = fft_smem_x(a), sy = fft_smem_yz(a, a.ny), sz = fft_smem_yz(a, a.nz);
    cudaError_t e;
    if ((e = set_smem(k_fft_x_fwd<T>, sx)) != cudaSuccess) return e;
    if ((e = set_smem(k_fft_x_inv<T>, sx)) != cudaSuccess) return e;
    if ((e = set_smem(k_fft_y<T, false>, sy)) != cudaSuccess) return e;
    if ((e = set_smem(k_fft_y<T, true>, sy)) != cudaSuccess) return e;
    return set_smem(k_fft_z_solve<T>, sz);
}

template <typename T>
cudaError_t Kernels<T>::poisson_iteration(const PoissonArgs<T>& a, cudaStream_t st, const LaunchHook* hook)
{
    const size_t sx = fft_smem_x(a), sy = fft_smem_yz(a, a.ny), sz = fft_smem_yz(a, a.nz);
    const int rows = a.ny * a.nz;
    const int gx = (rows + a.rows_per_block - 1) / a.rows_per_block;
    const int gc = (a.M + a.cols_per_block - 1) / a.cols_per_block;
    k_fft_x_fwd<T><<<gx, 256, sx, st>>>(a);
    if (hook) (*hook)(VF_PHASE_FFT_X_FWD);
    k_fft_y<T, false><<<dim3(gc, a.nz), 256, sy, st>>>(a);
    if (hook) (*hook)(VF_PHASE_FFT_Y_FWD);
    k_fft_z_solve<T><<<dim3(gc, a.ny), 256, sz, st>>>(a);
    if (hook) (*hook)(VF_PHASE_FFT_Z_SOLVE);
    k_fft_y<T, true><<<dim3(gc, a.nz), 256, sy, st>>>(a);
    if (hook) (*hook)(VF_PHASE_FFT_Y_INV);
    k_fft_x_inv<T><<<gx, 256, sx, st>>>(a);
    if (hook) (*hook)(VF_PHASE_FFT_X_INV);
    return cudaGetLastError();
}

template cudaError_t Kernels<float>::poisson_prepare(const PoissonArgs<float>&);
template cudaError_t Kernels<double>::poisson_prepare(const PoissonArgs<double>&);
template cudaError_t Kernels<float>::poisson_iteration(const PoissonArgs<float>&, cudaStream_t, const LaunchHook*);
template cudaError_t Kernels<double>::poisson_iteration(const PoissonArgs<double>&, cudaStream_t, const LaunchHook*);
template size_t Kernels<float>::fft_smem_x(const PoissonArgs<float>&);
template size_t Kernels<double>::fft_smem_x(const PoissonArgs<double>&);
template size_t Kernels<float>::fft_smem_yz(const PoissonArgs<float>&, int);
template size_t Kernels<double>::fft_smem_yz(const PoissonArgs<double>&, int);

}  // namespace vf
