// FFT Poisson solve of the pressure equation (Sec. 2.2, Eq. 9): p^{k+1} = L^{-1}[ D u*/dt + D((1 - beta) G p^k) ].
//
// One iteration:
//   correction : f = r + D((1 - beta) G p^k) at the listed cells that have a solid neighbour (elsewhere f = r);
//   x forward  : real-to-complex FFT of f along x (two real points packed per complex value, nx/2-point complex
//                FFT, then the split step);
//   then either (tile layout) y forward, z solve (z FFT, division by lambda N, inverse z FFT), y inverse, each a
//   pass over tiles of consecutive kx columns, or (plane layout) one pass in which a CTA per kx does the whole
//   (y, z) plane in shared memory;
//   x inverse  : complex-to-real inverse FFT along x, writes p^{k+1}.
// The spectrum has nx/2 complex columns per (y, z) row.  Column 0 holds the x-spectra at kx = 0 (real part)
// and kx = nx/2 (imaginary part): both are real for real data and both have sin^2(2 pi kx / nx) = 0, so the
// y/z transforms and the eigenvalue division treat the packed pair exactly like any other column.
//
// The transforms are mixed-radix (2, 3, 4, 5, 8, 16) Stockham FFTs: each radix pass is done by R-point butterflies
// in registers, passes exchange data through shared memory.  In the row and tile passes the first radix pass
// reads its operands straight from global memory and the last writes straight to its destination; the plane
// kernel works in place on one shared-memory plane (a barrier between the reads and the writes of each pass).
// Twiddles come from per-axis tables staged in shared memory; the index arithmetic uses precomputed
// multiply-shift divisions.
#include <cuda_runtime.h>

#include <cstdint>

#include "fft_common.cuh"

namespace vf {
namespace {

// One radix-R Stockham pass over nseq sequences.  Work item (j, b) reads element j + r nb of sequence b
// (r = 0..R-1), multiplies it by W_n^(r (j mod Ns) tstride), does a DFT of order R and writes element
// (j / Ns) Ns R + (j mod Ns) + r Ns.  ld(k, b) / st(k, b, v) access element k of sequence b.
// SEQFAST: consecutive threads take consecutive sequences (column tiles of TB); otherwise consecutive elements.
template <typename C, int R, bool INV, bool SEQFAST, int TB, typename LD, typename ST>
__device__ __forceinline__ void radix_pass(const FftStage& S, int nseq, const C* __restrict__ tw, LD ld, ST st)
{
    const int total = S.nb * nseq;
    for (int it = threadIdx.x; it < total; it += blockDim.x) {
        int j, b;
        if (SEQFAST) { b = it % TB; j = it / TB; }
        else { b = (int)fdiv((uint32_t)it, S.nb_div); j = it - b * S.nb; }
        const int jq = (int)fdiv((uint32_t)j, S.ns_div);
        const int jm = j - jq * S.Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = ld(j + r * S.nb, b);
        if (jm) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = tw[jm * r * S.tstride];
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft<C, R, INV>(v);
        const int d0 = jq * S.Ns * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) st(d0 + r * S.Ns, b, v[r]);
    }
}

template <typename C, bool INV, bool SEQFAST, int TB, typename LD, typename ST>
__device__ __forceinline__ void radix_pass_any(const FftStage& S, int nseq, const C* tw, LD ld, ST st)
{
    switch (S.R) {
        case 2: radix_pass<C, 2, INV, SEQFAST, TB>(S, nseq, tw, ld, st); break;
        case 3: radix_pass<C, 3, INV, SEQFAST, TB>(S, nseq, tw, ld, st); break;
        case 4: radix_pass<C, 4, INV, SEQFAST, TB>(S, nseq, tw, ld, st); break;
        case 5: radix_pass<C, 5, INV, SEQFAST, TB>(S, nseq, tw, ld, st); break;
        case 8: radix_pass<C, 8, INV, SEQFAST, TB>(S, nseq, tw, ld, st); break;
        default: radix_pass<C, 16, INV, SEQFAST, TB>(S, nseq, tw, ld, st); break;
    }
}

// Whole transform: pass 0 reads through `first`, the last pass writes through `last`, passes in between go
// through the shared buffers bufA / bufB (element k of sequence b at k * es + b * ss; pass 0 writes bufA).  The
// destination of `last` must be neither bufA nor bufB.  No barrier after the last pass.
template <typename C, bool INV, bool SEQFAST, int TB, typename FirstLD, typename LastST>
__device__ void fft_run(const FftAxis& ax, int nseq, int es, int ss, const C* tw, C* bufA, C* bufB, FirstLD first,
                        LastST last)
{
    C* src = bufB;
    C* dst = bufA;
    for (int s = 0; s < ax.nstages; ++s) {
        const FftStage& S = ax.st[s];
        // column tiles (SEQFAST): element k of column b at k * es + b; rows: padded element k of row b at b * ss
        auto sld = [src, es, ss](int k, int b) { return SEQFAST ? src[k * es + b] : src[b * ss + padded(k)]; };
        auto sst = [dst, es, ss](int k, int b, C v) {
            if (SEQFAST) dst[k * es + b] = v;
            else dst[b * ss + padded(k)] = v;
        };
        const bool is_first = s == 0, is_last = s == ax.nstages - 1;
        if (is_first && is_last) radix_pass_any<C, INV, SEQFAST, TB>(S, nseq, tw, first, last);
        else if (is_first) radix_pass_any<C, INV, SEQFAST, TB>(S, nseq, tw, first, sst);
        else if (is_last) radix_pass_any<C, INV, SEQFAST, TB>(S, nseq, tw, sld, last);
        else radix_pass_any<C, INV, SEQFAST, TB>(S, nseq, tw, sld, sst);
        if (!is_last) {
            __syncthreads();
            src = dst;
            dst = (dst == bufA) ? bufB : bufA;
        }
    }
}

// f = r + correction at every listed cell; the first iteration of a step also saves r there (f holds r then)
template <typename T>
__global__ void __launch_bounds__(256) k_poisson_correction(PoissonArgs<T> A, int first)
{
    pdl_enter();
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < A.n_near; j += gridDim.x * blockDim.x) {
        const int i = __ldg(A.near_list + j);
        const int t = (int)fdiv((uint32_t)i, A.nx_div), x = i - t * A.nx;
        const int z = (int)fdiv((uint32_t)t, A.ny_div), y = t - z * A.ny;
        T rr;
        if (first) {
            rr = A.f[i];
            A.near_r[j] = rr;
        } else {
            rr = A.near_r[j];
        }
        A.f[i] = rr + poisson_correction(A, i, x, y, z);
    }
}

// ---- x forward: real-to-complex FFT of f along x -----------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_fft_x_fwd(PoissonArgs<T> A)
{
    pdl_enter();
    using C = typename CxT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = A.M, B = A.rows_per_block;
    C* tw = reinterpret_cast<C*>(smem_raw);
    const int SS = padded_stride(M);
    C* bufA = tw + M;
    C* bufB = bufA + B * SS;
    C* out = bufB + B * SS;
    stage_table(tw, A.twx, M);
    const int rows = A.ny * A.nz;
    const int row0 = blockIdx.x * B;
    // element k of row b: (f[2k], f[2k+1])
    auto first = [&](int k, int b) -> C {
        const int row = row0 + b;
        if (row >= rows) return mk<C>(T(0), T(0));
        return *reinterpret_cast<const C*>(A.f + (long long)row * A.nx + 2 * k);
    };
    auto last = [&](int k, int b, C v) { out[b * SS + padded(k)] = v; };
    __syncthreads();
    fft_run<C, false, false, 1>(A.ax, B, 1, SS, tw, bufA, bufB, first, last);
    __syncthreads();
    const C* twr = reinterpret_cast<const C*>(A.twr);
    C* spec = reinterpret_cast<C*>(A.spec);
    for (int it = threadIdx.x; it < B * M; it += blockDim.x) {
        // plane layout: consecutive threads take consecutive rows of one kx (coalesced writes)
        int b, k;
        if (A.plane_layout) { k = it / B; b = it - k * B; }
        else { b = it / M; k = it - b * M; }
        const int row = row0 + b;
        if (row >= rows) continue;
        const C Zk = out[b * SS + padded(k)];
        C X;
        if (k == 0) {
            X = mk<C>(Zk.x + Zk.y, Zk.x - Zk.y);                 // (X_0, X_{nx/2})
        } else {
            const C Zm = out[b * SS + padded(M - k)];           // conj taken below
            const C E = mk<C>(T(0.5) * (Zk.x + Zm.x), T(0.5) * (Zk.y - Zm.y));
            const C O = mk<C>(T(0.5) * (Zk.y + Zm.y), T(-0.5) * (Zk.x - Zm.x));
            X = cadd(E, cmul(__ldg(&twr[k]), O));               // X_k = E_k + W^k O_k
        }
        if (A.plane_layout) spec[(long long)k * rows + row] = X;
        else spec[(long long)row * M + k] = X;
    }
}

// ---- y pass (forward or inverse), in place on the spectrum --------------------------------------------------
template <typename T, bool INV, int TB>
__global__ void __launch_bounds__(256) k_fft_y(PoissonArgs<T> A)
{
    pdl_enter();
    using C = typename CxT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = A.ny, M = A.M;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* bufA = tw + n;
    C* bufB = bufA + TB * n;
    stage_table(tw, A.twy, n);
    const int kx0 = blockIdx.x * TB;
    C* spec = reinterpret_cast<C*>(A.spec) + (long long)blockIdx.y * n * M + kx0;
    const bool full = kx0 + TB <= M;
    auto first = [&](int y, int b) -> C {
        return (full || kx0 + b < M) ? spec[(long long)y * M + b] : mk<C>(T(0), T(0));
    };
    auto last = [&](int y, int b, C v) {
        if (full || kx0 + b < M) spec[(long long)y * M + b] = v;
    };
    __syncthreads();
    fft_run<C, INV, true, TB>(A.ay, TB, TB, 1, tw, bufA, bufB, first, last);
}

// ---- z pass: forward FFT, division by the Laplacian eigenvalues, inverse FFT --------------------------------
template <typename T, int TB>
__global__ void __launch_bounds__(256) k_fft_z_solve(PoissonArgs<T> A)
{
    pdl_enter();
    using C = typename CxT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = A.nz, M = A.M, ny = A.ny;
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* bufA = tw + n;
    C* bufB = bufA + TB * n;
    C* mid = bufB + TB * n;
    stage_table(tw, A.twz, n);
    const int kx0 = blockIdx.x * TB;
    const int ky = blockIdx.y;
    const long long zstride = (long long)ny * M;
    C* spec = reinterpret_cast<C*>(A.spec) + (long long)ky * M + kx0;
    const bool full = kx0 + TB <= M;
    const T ly = __ldg(A.lamy + ky);
    const bool ky_null = (ky == 0) || (2 * ky == ny);
    auto gload = [&](int z, int b) -> C {
        return (full || kx0 + b < M) ? spec[z * zstride + b] : mk<C>(T(0), T(0));
    };
    // the forward result is scaled by 1 / (lambda N) on its way into shared memory
    auto scaled_store = [&](int kz, int b, C v) {
        const int kx = kx0 + b;
        T s = T(0);
        if (kx < M) {
            const bool null = (kx == 0) && ky_null && ((kz == 0) || (2 * kz == n));
            if (!null) s = inv_lambda(A.invN, __ldg(A.lamx + kx) + ly + __ldg(A.lamz + kz));
        }
        mid[kz * TB + b] = cscale(v, s);
    };
    auto sload = [&](int kz, int b) -> C { return mid[kz * TB + b]; };
    auto gstore = [&](int z, int b, C v) {
        if (full || kx0 + b < M) spec[z * zstride + b] = v;
    };
    __syncthreads();
    fft_run<C, false, true, TB>(A.az, TB, TB, 1, tw, bufA, bufB, gload, scaled_store);
    __syncthreads();
    fft_run<C, true, true, TB>(A.az, TB, TB, 1, tw, bufA, bufB, sload, gstore);
}

// ---- x inverse: complex-to-real FFT along x, writes p ---------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_fft_x_inv(PoissonArgs<T> A)
{
    pdl_enter();
    using C = typename CxT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = A.M, B = A.rows_per_block;
    C* tw = reinterpret_cast<C*>(smem_raw);
    const int SS = padded_stride(M);
    C* bufA = tw + M;
    C* bufB = bufA + B * SS;
    C* in = bufB + B * SS;
    stage_table(tw, A.twx, M);
    const int rows = A.ny * A.nz;
    const int row0 = blockIdx.x * B;
    const C* spec = reinterpret_cast<const C*>(A.spec);
    const C* twr = reinterpret_cast<const C*>(A.twr);
    if (A.plane_layout) {
        // stage the block's rows in shared memory with coalesced reads (consecutive rows of one kx), 8 loads in
        // flight per thread
        for (int it0 = threadIdx.x; it0 < B * M; it0 += 8 * blockDim.x) {
            C tmp[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int it = it0 + u * blockDim.x;
                const int k = it / B, b = it - k * B, row = row0 + b;
                tmp[u] = (it < B * M && row < rows) ? spec[(long long)k * rows + row] : mk<C>(T(0), T(0));
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int it = it0 + u * blockDim.x;
                if (it < B * M) {
                    const int k = it / B, b = it - k * B;
                    in[b * SS + padded(k)] = tmp[u];
                }
            }
        }
    }
    auto spec_at = [&](int k, int b) -> C {
        return A.plane_layout ? in[b * SS + padded(k)] : spec[(long long)(row0 + b) * M + k];
    };
    // element k of the half-length sequence: Z'_k = (X_k + conj X_{M-k}) + i W^{-k} (X_k - conj X_{M-k})
    auto first = [&](int k, int b) -> C {
        const int row = row0 + b;
        if (row >= rows) return mk<C>(T(0), T(0));
        const C Xk = spec_at(k, b);
        if (k == 0) return mk<C>(Xk.x + Xk.y, Xk.x - Xk.y);
        const C Xm = spec_at(M - k, b);
        const C s = mk<C>(Xk.x + Xm.x, Xk.y - Xm.y);
        const C d = mk<C>(Xk.x - Xm.x, Xk.y + Xm.y);
        C w = __ldg(&twr[k]);
        w.y = -w.y;
        const C wd = cmul(w, d);
        return mk<C>(s.x - wd.y, s.y + wd.x);
    };
    auto last = [&](int k, int b, C v) {
        const int row = row0 + b;
        if (row < rows) *reinterpret_cast<C*>(A.p + (long long)row * A.nx + 2 * k) = v;
    };
    __syncthreads();
    fft_run<C, true, false, 1>(A.ax, B, 1, SS, tw, bufA, bufB, first, last);
}

// ---- plane layout: the whole (y, z) plane of one kx, in place in shared memory ------------------------------
// Forward transforms are in-place decimation-in-frequency passes (each butterfly writes back to the positions it
// read, so a pass needs no barrier between its reads and writes); they leave the spectrum in digit-reversed
// order, which the eigenvalue division reads through the krev tables.  The inverse transforms are the mirrored
// decimation-in-time passes, which take the digit-reversed spectrum back to natural order.
// Element e of sequence b is at e * es + b * ss.  SEQFAST: consecutive threads take consecutive sequences.
template <typename C, int R, bool INV, bool SEQFAST, typename IDX>
__device__ __forceinline__ void inplace_pass(C* buf, const FftStage& S, int nseq, const FastDiv& nseq_div, IDX idx,
                                             const C* __restrict__ tw)
{
    const int per_seq = S.nb;                 // butterflies per sequence (n / R)
    const int total = per_seq * nseq;
    const int m = S.tstride;                  // group stride L / R
    for (int it = threadIdx.x; it < total; it += blockDim.x) {
        int w, b;
        if (SEQFAST) { w = (int)fdiv((uint32_t)it, nseq_div); b = it - w * nseq; }
        else { b = (int)fdiv((uint32_t)it, S.nb_div); w = it - b * per_seq; }
        const int blk = (int)fdiv((uint32_t)w, S.m_div);
        const int j = w - blk * m;
        const int base = blk * m * R + j;     // block start (blk * L) + j
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = buf[idx(base + r * m, b)];
        if (!INV) {
            dft<C, R, false>(v);
            if (j) {
#pragma unroll
                for (int k = 1; k < R; ++k) v[k] = cmul(v[k], tw[j * k * S.Ns]);
            }
        } else {
            if (j) {
#pragma unroll
                for (int k = 1; k < R; ++k) {
                    C t = tw[j * k * S.Ns];
                    t.y = -t.y;
                    v[k] = cmul(v[k], t);
                }
            }
            dft<C, R, true>(v);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) buf[idx(base + r * m, b)] = v[r];
    }
    __syncthreads();
}

// all radix passes of one axis; idx(e, b) is the shared-memory slot of element e of sequence b
template <typename C, bool INV, bool SEQFAST, typename IDX>
__device__ void inplace_fft(C* buf, const FftAxis& ax, int nseq, const FastDiv& nseq_div, IDX idx, const C* tw)
{
    for (int i = 0; i < ax.nstages; ++i) {
        const int s = INV ? ax.nstages - 1 - i : i;   // the inverse runs the stages in reverse order
        const FftStage& S = ax.st[s];
        switch (S.R) {
            case 2: inplace_pass<C, 2, INV, SEQFAST>(buf, S, nseq, nseq_div, idx, tw); break;
            case 3: inplace_pass<C, 3, INV, SEQFAST>(buf, S, nseq, nseq_div, idx, tw); break;
            case 4: inplace_pass<C, 4, INV, SEQFAST>(buf, S, nseq, nseq_div, idx, tw); break;
            case 5: inplace_pass<C, 5, INV, SEQFAST>(buf, S, nseq, nseq_div, idx, tw); break;
            case 8: inplace_pass<C, 8, INV, SEQFAST>(buf, S, nseq, nseq_div, idx, tw); break;
            default: inplace_pass<C, 16, INV, SEQFAST>(buf, S, nseq, nseq_div, idx, tw); break;
        }
    }
}

// plane [z][y] of one kx (row z at z * SP, element y at padded(y)): y FFT (rows), z FFT (columns),
// x 1 / (lambda N), inverse z FFT, inverse y FFT
template <typename T>
__global__ void __launch_bounds__(kPlaneThreads) k_fft_yz_solve(PoissonArgs<T> A)
{
    pdl_enter();
    using C = typename CxT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ny = A.ny, nz = A.nz, n_el = ny * nz;
    const int SP = padded_stride(ny);
    C* plane = reinterpret_cast<C*>(smem_raw);
    C* twy = plane + (size_t)SP * nz;
    C* twz = twy + ny;
    int* ky_of = reinterpret_cast<int*>(twz + nz);
    int* kz_of = ky_of + ny;
    const int kx = blockIdx.x;
    C* g = reinterpret_cast<C*>(A.spec) + (long long)kx * n_el;
    // load the plane 8 values per thread at a time, so the global loads of a thread overlap
    for (int i0 = threadIdx.x; i0 < n_el; i0 += 8 * kPlaneThreads) {
        C tmp[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * kPlaneThreads;
            if (i < n_el) tmp[u] = g[i];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * kPlaneThreads;
            if (i < n_el) {
                const int z = (int)fdiv((uint32_t)i, A.ny_div), y = i - z * ny;
                plane[z * SP + padded(y)] = tmp[u];
            }
        }
    }
    stage_table(twy, A.twy, ny);
    stage_table(twz, A.twz, nz);
    for (int i = threadIdx.x; i < ny; i += blockDim.x) ky_of[i] = __ldg(A.krev_y + i);
    for (int i = threadIdx.x; i < nz; i += blockDim.x) kz_of[i] = __ldg(A.krev_z + i);
    const FastDiv nz_div = make_fast_div_dev(nz);
    auto row_idx = [SP](int e, int b) { return b * SP + padded(e); };   // element e = y of row b = z
    auto col_idx = [SP](int e, int b) { return e * SP + padded(b); };   // element e = z of column b = y
    __syncthreads();
    inplace_fft<C, false, false>(plane, A.ay, nz, nz_div, row_idx, twy);
    inplace_fft<C, false, true>(plane, A.az, ny, A.ny_div, col_idx, twz);
    const T lx = __ldg(A.lamx + kx);
    for (int i = threadIdx.x; i < n_el; i += blockDim.x) {
        const int pz = (int)fdiv((uint32_t)i, A.ny_div), py = i - pz * ny;
        const int ky = ky_of[py], kz = kz_of[pz];
        const bool null = (kx == 0) && (ky == 0 || 2 * ky == ny) && (kz == 0 || 2 * kz == nz);
        const T s = null ? T(0) : inv_lambda(A.invN, lx + __ldg(A.lamy + ky) + __ldg(A.lamz + kz));
        const int q = pz * SP + padded(py);
        plane[q] = cscale(plane[q], s);
    }
    __syncthreads();
    inplace_fft<C, true, true>(plane, A.az, ny, A.ny_div, col_idx, twz);
    inplace_fft<C, true, false>(plane, A.ay, nz, nz_div, row_idx, twy);
    for (int i = threadIdx.x; i < n_el; i += blockDim.x) {
        const int z = (int)fdiv((uint32_t)i, A.ny_div), y = i - z * ny;
        g[i] = plane[z * SP + padded(y)];
    }
}

// The dynamic shared-memory limit is a per-kernel, process-wide attribute: it is raised to the device's opt-in
// maximum (an upper bound only; each launch uses its own size), never lowered, so grids of different sizes can
// be created in any order.
template <typename K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (bytes > (size_t)optin) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

template <typename T> constexpr int cols_tb() { return sizeof(T) == 8 ? 8 : 16; }

}  // namespace

template <typename T>
bool Kernels<T>::plane_fits(int ny, int nz)
{
    const size_t bytes = ((size_t)padded_stride(ny) * nz + ny + nz) * sizeof(typename CxT<T>::type) +
                         (size_t)(ny + nz) * sizeof(int);
    return bytes <= 200 * 1024;
}

template <typename T>
size_t Kernels<T>::fft_smem_x(const PoissonArgs<T>& a)
{
    // twiddle table + two exchange buffers + the output of the last pass (x forward) / staged input (x inverse)
    return (3 * (size_t)a.rows_per_block * padded_stride(a.M) + a.M) * sizeof(typename CxT<T>::type);
}

template <typename T>
size_t Kernels<T>::fft_smem_yz(const PoissonArgs<T>& a, int n, int buffers)
{
    // twiddle table + exchange buffers (y: 2; z solve: 2 + the scaled forward result)
    return ((size_t)buffers * cols_tb<T>() * n + n) * sizeof(typename CxT<T>::type);
}

template <typename T>
size_t Kernels<T>::fft_smem_plane(const PoissonArgs<T>& a)
{
    return ((size_t)padded_stride(a.ny) * a.nz + a.ny + a.nz) * sizeof(typename CxT<T>::type) +
           (size_t)(a.ny + a.nz) * sizeof(int);
}

template <typename T>
cudaError_t Kernels<T>::poisson_prepare(const PoissonArgs<T>& a)
{
    if (a.reg) return RegFft<T>::prepare(a);
    constexpr int TB = cols_tb<T>();
    const size_t sx = fft_smem_x(a), sy = fft_smem_yz(a, a.ny, 2), sz = fft_smem_yz(a, a.nz, 3);
    cudaError_t e;
    if ((e = set_smem(k_fft_x_fwd<T>, sx)) != cudaSuccess) return e;
    if ((e = set_smem(k_fft_x_inv<T>, sx)) != cudaSuccess) return e;
    if (a.plane_layout) return set_smem(k_fft_yz_solve<T>, fft_smem_plane(a));
    if ((e = set_smem(k_fft_y<T, false, TB>, sy)) != cudaSuccess) return e;
    if ((e = set_smem(k_fft_y<T, true, TB>, sy)) != cudaSuccess) return e;
    return set_smem(k_fft_z_solve<T, TB>, sz);
}

template <typename T>
cudaError_t Kernels<T>::poisson_iteration(const PoissonArgs<T>& a, int first, cudaStream_t st,
                                          const LaunchHook* hook)
{
    if (a.n_near > 0) {
        const int gb = (a.n_near + 255) / 256;
        const cudaError_t e = launch_pdl(k_poisson_correction<T>, dim3(gb < 4096 ? gb : 4096), dim3(256), 0, st, a,
                                         first);
        if (e != cudaSuccess) return e;
        if (hook) (*hook)(VF_PHASE_POISSON_RHS);
    }
    if (a.reg) return RegFft<T>::iteration(a, st, hook);
    constexpr int TB = cols_tb<T>();
    if (a.cols_per_block != TB) return cudaErrorInvalidValue;
    const size_t sx = fft_smem_x(a);
    const int rows = a.ny * a.nz;
    const int gx = (rows + a.rows_per_block - 1) / a.rows_per_block;
    cudaError_t e;
    if ((e = launch_pdl(k_fft_x_fwd<T>, dim3(gx), dim3(256), sx, st, a)) != cudaSuccess) return e;
    if (hook) (*hook)(VF_PHASE_FFT_X_FWD);
    if (a.plane_layout) {
        if ((e = launch_pdl(k_fft_yz_solve<T>, dim3(a.M), dim3(kPlaneThreads), fft_smem_plane(a), st, a)) !=
            cudaSuccess)
            return e;
        if (hook) (*hook)(VF_PHASE_FFT_YZ_SOLVE);
    } else {
        const size_t sy = fft_smem_yz(a, a.ny, 2), sz = fft_smem_yz(a, a.nz, 3);
        const int gc = (a.M + TB - 1) / TB;
        if ((e = launch_pdl(k_fft_y<T, false, TB>, dim3(gc, a.nz), dim3(256), sy, st, a)) != cudaSuccess) return e;
        if (hook) (*hook)(VF_PHASE_FFT_Y_FWD);
        if ((e = launch_pdl(k_fft_z_solve<T, TB>, dim3(gc, a.ny), dim3(256), sz, st, a)) != cudaSuccess) return e;
        if (hook) (*hook)(VF_PHASE_FFT_Z_SOLVE);
        if ((e = launch_pdl(k_fft_y<T, true, TB>, dim3(gc, a.nz), dim3(256), sy, st, a)) != cudaSuccess) return e;
        if (hook) (*hook)(VF_PHASE_FFT_Y_INV);
    }
    if ((e = launch_pdl(k_fft_x_inv<T>, dim3(gx), dim3(256), sx, st, a)) != cudaSuccess) return e;
    if (hook) (*hook)(VF_PHASE_FFT_X_INV);
    return cudaSuccess;
}

template cudaError_t Kernels<float>::poisson_prepare(const PoissonArgs<float>&);
template cudaError_t Kernels<double>::poisson_prepare(const PoissonArgs<double>&);
template cudaError_t Kernels<float>::poisson_iteration(const PoissonArgs<float>&, int, cudaStream_t, const LaunchHook*);
template cudaError_t Kernels<double>::poisson_iteration(const PoissonArgs<double>&, int, cudaStream_t, const LaunchHook*);
template bool Kernels<float>::plane_fits(int, int);
template bool Kernels<double>::plane_fits(int, int);
template size_t Kernels<float>::fft_smem_plane(const PoissonArgs<float>&);
template size_t Kernels<double>::fft_smem_plane(const PoissonArgs<double>&);
template size_t Kernels<float>::fft_smem_x(const PoissonArgs<float>&);
template size_t Kernels<double>::fft_smem_x(const PoissonArgs<double>&);
template size_t Kernels<float>::fft_smem_yz(const PoissonArgs<float>&, int, int);
template size_t Kernels<double>::fft_smem_yz(const PoissonArgs<double>&, int, int);

}  // namespace vf
