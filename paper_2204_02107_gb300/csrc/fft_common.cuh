// Device helpers shared by the FFT Poisson kernels: complex arithmetic, small DFTs in registers (orders 2, 3,
// 4, 5, 8, 16), shared-memory row padding, multiply-shift division, table staging and the Eq. 9 correction
// D((1 - beta) G p) at one cell.  Included by the kernel files only (everything has internal linkage).
#pragma once

#include <utility>
#include <cuda_runtime.h>

#include <cstdint>

#include "launch.cuh"
#include "vf_internal.h"

namespace vf {
namespace {

template <typename T> struct CxT;
template <> struct CxT<float> { using type = float2; };
template <> struct CxT<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) { C r; r.x = a; r.y = b; return r; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
#ifndef VF_NO_PACKED_F32
// FP32 complex add and subtract as one packed two-lane instruction each (a - b = fma(b, -1, a), exact)
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
#endif
template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
// multiply by +i (INV) or -i (forward): the rotation of a forward / inverse DFT of order 4
template <typename C, bool INV> __device__ __forceinline__ C rot(C a) { return INV ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x); }

// Shared-memory row layout of the row passes and the plane: one padding element per 16 complex values inside a
// row and an odd row stride, so the strided writes of a radix pass and the row-crossing reads of the split steps
// spread over the banks.
__host__ __device__ __forceinline__ int padded(int e) { return e + (e >> 4); }
__host__ __device__ __forceinline__ int padded_stride(int n) { return (padded(n - 1) + 1) | 1; }

__device__ __forceinline__ FastDiv make_fast_div_dev(uint32_t d)
{
    FastDiv f{d, 0u, 0u};
    if (d <= 1) return f;
    uint32_t l = 32 - __clz(d - 1);   // ceil(log2 d)
    f.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
    f.s = l;
    return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f)
{
    if (f.d <= 1) return n;
    const uint32_t t = __umulhi(f.m, n);
    return (t + ((n - t) >> 1)) >> (f.s - 1);
}

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

// order 16 as 4 x 4: DFT4 over the stride-4 columns, twiddles W16^(n2 k1), DFT4 over the rows, transpose
template <typename C, bool INV>
__device__ __forceinline__ void dft16(C* v)
{
    using R = decltype(C::x);
    const R c1 = R(0.92387953251128675613), s1 = R(0.38268343236508977173), h = R(0.70710678118654752440);
    const R sg = INV ? R(1) : R(-1);   // sign of the imaginary part of W16^k
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<C, INV>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    const C w1 = mk<C>(c1, sg * s1), w2 = mk<C>(h, sg * h), w3 = mk<C>(s1, sg * c1);
    const C w6 = mk<C>(-h, sg * h), w9 = mk<C>(-c1, -sg * s1);
    v[5] = cmul(v[5], w1); v[9] = cmul(v[9], w2); v[13] = cmul(v[13], w3);
    v[6] = cmul(v[6], w2); v[10] = rot<C, INV>(v[10]); v[14] = cmul(v[14], w6);
    v[7] = cmul(v[7], w3); v[11] = cmul(v[11], w6); v[15] = cmul(v[15], w9);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<C, INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    C t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
}

template <typename C, int R, bool INV>
__device__ __forceinline__ void dft(C* v);

// f(std::integral_constant<int, i>) for i = 0 .. N-1, expanded at compile time
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---- composite orders: compile-time Cooley-Tukey split R = A B in registers ---------------------------------
// cos and sin of 2 pi j / n evaluated at compile time (argument reduced to [-pi/4, pi/4] by octant, then Taylor
// series to 1e-17), for the constant twiddles of the composite small DFTs
constexpr double kTwoPi = 6.283185307179586476925286766559;
__host__ __device__ constexpr double taylor_sin(double x)
{
    double term = x, sum = x;
    for (int k = 1; k < 14; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double taylor_cos(double x)
{
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 14; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
// (cos, sin) of 2 pi j / n: j / n reduced to eighths of a turn
__host__ __device__ constexpr double cos_turn(long long j, long long n)
{
    j %= n;
    if (j < 0) j += n;
    const long long o = (8 * j) / n;                           // octant 0..7
    const double r = kTwoPi * ((double)(8 * j - o * n) / (8.0 * n));   // remainder angle in [0, pi/4)
    const double c = taylor_cos(r), s = taylor_sin(r);
    // cos(o pi/4 + r) for o = 0..7 with the 45-degree rotations written out
    constexpr double h = 0.70710678118654752440;
    switch (o) {
        case 0: return c;
        case 1: return h * (c - s);
        case 2: return -s;
        case 3: return -h * (c + s);
        case 4: return -c;
        case 5: return -h * (c - s);
        case 6: return s;
        default: return h * (c + s);
    }
}

// first factor of a composite order (the remaining factor is R / factor)
template <int R> __host__ __device__ constexpr int ct_factor()
{
    return R % 16 == 0 && R > 16 ? 16 : R % 8 == 0 && R > 8 ? 8 : R % 4 == 0 && R > 4 ? 4 : R % 2 == 0 && R > 2 ? 2 :
           R % 3 == 0 && R > 3 ? 3 : R % 5 == 0 && R > 5 ? 5 : R;
}

// X[k1 + A k2] = sum_b W_B^(b k2) W_R^(b k1) sum_a x[b + B a] W_A^(a k1): DFTs of order A over a, the twiddles,
// DFTs of order B over b; in place, natural order in and out
template <typename C, int A, int B, bool INV>
__device__ __forceinline__ void dft_ct(C* v)
{
    using T = decltype(C::x);
    constexpr int R = A * B;
    C y[B][A];
#pragma unroll
    for (int b = 0; b < B; ++b) {
#pragma unroll
        for (int a = 0; a < A; ++a) y[b][a] = v[b + B * a];
        dft<C, A, INV>(y[b]);
    }
    // W_R^(b k1) = exp(-+ 2 pi i b k1 / R), each a compile-time constant
    static_for<B * A>([&](auto I) {
        constexpr int b = decltype(I)::value / A, k1 = decltype(I)::value % A;
        if constexpr (b > 0 && k1 > 0) {
            constexpr double c = cos_turn((long long)b * k1, R);
            constexpr double sn = (INV ? 1.0 : -1.0) * cos_turn((long long)b * k1 * 4 - R, 4LL * R);
            y[b][k1] = cmul(y[b][k1], mk<C>((T)c, (T)sn));
        }
    });
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
        C z[B];
#pragma unroll
        for (int b = 0; b < B; ++b) z[b] = y[b][k1];
        dft<C, B, INV>(z);
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = z[k2];
    }
}

template <typename C, int R, bool INV>
__device__ __forceinline__ void dft(C* v)
{
    if constexpr (R == 1) {
    } else if constexpr (R == 2) dft2<C, INV>(v[0], v[1]);
    else if constexpr (R == 3) dft3<C, INV>(v[0], v[1], v[2]);
    else if constexpr (R == 4) dft4<C, INV>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 5) dft5<C, INV>(v[0], v[1], v[2], v[3], v[4]);
    else if constexpr (R == 8) dft8<C, INV>(v);
    else if constexpr (R == 16) dft16<C, INV>(v);
    else dft_ct<C, ct_factor<R>(), R / ct_factor<R>(), INV>(v);
}

// 1 / (lambda N) factor of the eigenvalue division, -invN / sum: in FP32 the fast division (two multiplies by an
// approximate reciprocal, within 2 ulp), in FP64 the correctly rounded one
__device__ __forceinline__ float inv_lambda(float invN, float sum) { return __fdividef(-invN, sum); }
__device__ __forceinline__ double inv_lambda(double invN, double sum) { return -invN / sum; }

template <typename C>
__device__ __forceinline__ void stage_table(C* dst, const void* src, int n)
{
    const C* s = reinterpret_cast<const C*>(src);
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = __ldg(s + i);
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Eq. 9 correction at one cell: sum_j (1/(2h_j))^2 [(1 - beta^+)(p^{++} - p^0) - (1 - beta^-)(p^0 - p^{--})]
// (= sum_j delta_j((1 - beta) delta_j p) with central differences).  Only called for cells with a solid neighbour.
// The betas of the six axis neighbours come from the cell's packed stencil-mask byte; p two cells away is loaded
// only along the directions whose neighbour is solid (the other terms are zero), all loads issued before any use.
template <typename T>
__device__ T poisson_correction(const PoissonArgs<T>& A, int i, int x, int y, int z)
{
    const int nx = A.nx, plane = A.nx * A.ny;
    const uint8_t sm = __ldg(A.smask + i);
    const bool sxm = !(sm & kSmXm), sxp = !(sm & kSmXp), sym = !(sm & kSmYm), syp = !(sm & kSmYp);
    const bool szm = !(sm & kSmZm), szp = !(sm & kSmZp);   // neighbour solid
    const T p0 = __ldg(A.p + i);
    T pxm = T(0), pxp = T(0), pym = T(0), pyp = T(0), pzm = T(0), pzp = T(0);
    if (sxm) pxm = __ldg(A.p + i - x + wrapi(x - 2, A.nx));
    if (sxp) pxp = __ldg(A.p + i - x + wrapi(x + 2, A.nx));
    if (sym) pym = __ldg(A.p + i + (wrapi(y - 2, A.ny) - y) * nx);
    if (syp) pyp = __ldg(A.p + i + (wrapi(y + 2, A.ny) - y) * nx);
    if (szm) pzm = __ldg(A.p + i + (wrapi(z - 2, A.nz) - z) * plane);
    if (szp) pzp = __ldg(A.p + i + (wrapi(z + 2, A.nz) - z) * plane);
    T corr = T(0);
    {
        const T pp = sxp ? pxp - p0 : T(0);
        const T pm = sxm ? p0 - pxm : T(0);
        corr += A.i2h2[0] * (pp - pm);
    }
    {
        const T pp = syp ? pyp - p0 : T(0);
        const T pm = sym ? p0 - pym : T(0);
        corr += A.i2h2[1] * (pp - pm);
    }
    {
        const T pp = szp ? pzp - p0 : T(0);
        const T pm = szm ? p0 - pzm : T(0);
        corr += A.i2h2[2] * (pp - pm);
    }
    return corr;
}

}  // namespace
}  // namespace vf
