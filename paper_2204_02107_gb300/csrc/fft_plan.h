// Radix schedules of one FFT axis of the generic mixed-radix passes, for the autotuner (host code only).
//
// A length n = 2^t 3^a 5^b can be transformed by any ordered list of radices from {2, 3, 4, 5, 8, 16} whose
// product is n; the generic kernels take the list at run time (each pass reads its radix from FftStage), and the
// in-place (y, z) plane kernel's digit-reversal tables follow the list.  Which list is fastest depends on the
// length, the pass (row, column tile or plane) and the precision, so the autotuner times a few of them.
// Candidate 0 is make_fft_axis's own schedule; the others vary the split of the power-of-two part (as many
// radix-16, radix-8 or radix-4 passes as possible, or the default split with its small radices first) and put
// the odd factors last or first; power-of-two parts of at most 8 also try radix-2 passes.  Every schedule computes
// the same DFT; only the rounding order differs.
#pragma once

#include <algorithm>
#include <vector>

#include "vf_internal.h"

namespace vf {

constexpr int kMaxFftSchedules = 8;

// Candidate radix lists of length n, candidate 0 first; empty if n is not 2-3-5 smooth or n < 2.
inline std::vector<std::vector<int>> fft_schedules(int n)
{
    std::vector<std::vector<int>> out;
    if (n < 2) return out;
    int m = n, t = 0, a = 0, b = 0;
    while (m % 2 == 0) { m /= 2; ++t; }
    while (m % 3 == 0) { m /= 3; ++a; }
    while (m % 5 == 0) { m /= 5; ++b; }
    if (m != 1) return out;

    const FftAxis d = make_fft_axis(n);
    std::vector<int> def_pow2;
    for (int s = 0; s < d.nstages; ++s)
        if (d.st[s].R != 3 && d.st[s].R != 5) def_pow2.push_back(d.st[s].R);
    // as many passes of radix 2^e as possible, the remainder (one smaller power of two) last
    auto greedy = [t](int e) {
        std::vector<int> r;
        int left = t;
        while (left >= e) { r.push_back(1 << e); left -= e; }
        if (left > 0) r.push_back(1 << left);
        return r;
    };
    std::vector<int> rev_pow2(def_pow2.rbegin(), def_pow2.rend());
    std::vector<std::vector<int>> pow2s = {def_pow2, greedy(4), greedy(3), greedy(2), rev_pow2};
    if (t <= 3) pow2s.push_back(greedy(1));   // radix-2 passes only for short power-of-two parts
    std::vector<int> odd;
    for (int i = 0; i < a; ++i) odd.push_back(3);
    for (int i = 0; i < b; ++i) odd.push_back(5);

    for (int odd_first = 0; odd_first < 2; ++odd_first) {
        for (const std::vector<int>& p2 : pow2s) {
            std::vector<int> r;
            if (odd_first) r.insert(r.end(), odd.begin(), odd.end());
            r.insert(r.end(), p2.begin(), p2.end());
            if (!odd_first) r.insert(r.end(), odd.begin(), odd.end());
            if ((int)r.size() > kMaxRadixStages) continue;
            if (std::find(out.begin(), out.end(), r) != out.end()) continue;
            if ((int)out.size() < kMaxFftSchedules) out.push_back(r);
        }
    }
    return out;
}

// The axis of length n with candidate schedule `index` (0: make_fft_axis(n)).  Stage s of a list R_0, R_1, ...
// has Ns = R_0 ... R_{s-1}, nb = n / R_s and twiddle stride n / (Ns R_s), as in make_fft_axis.  An index outside
// the candidates gives candidate 0.
inline FftAxis make_fft_axis_sched(int n, int index)
{
    if (index == 0) return make_fft_axis(n);
    const std::vector<std::vector<int>> c = fft_schedules(n);
    if (index < 0 || index >= (int)c.size()) return make_fft_axis(n);
    const std::vector<int>& rad = c[index];
    FftAxis ax{};
    ax.n = n;
    ax.nstages = (int)rad.size();
    int Ns = 1;
    for (int s = 0; s < ax.nstages; ++s) {
        FftStage& S = ax.st[s];
        S.R = rad[s];
        S.Ns = Ns;
        S.nb = n / S.R;
        S.tstride = n / (Ns * S.R);
        S.ns_div = make_fast_div((uint32_t)Ns);
        S.nb_div = make_fast_div((uint32_t)S.nb);
        S.m_div = make_fast_div((uint32_t)S.tstride);
        Ns *= S.R;
    }
    return ax;
}

}  // namespace vf
