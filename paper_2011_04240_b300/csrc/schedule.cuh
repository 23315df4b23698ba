// Multiplier layout and pair schedule of the pair step (shared by the
// batched pair kernels and the one-block-per-instance solver).
//
// Agents are padded to nbk blocks of G; a warp lane l of lane row tr handles
// agent l of a block and two samples (tsel) of a time block of 64/G samples.
// Per time block the steps sg enumerate, block row by block row, the G/2
// diagonal steps (partner (l + s) mod G, s = 1..G/2) and the G steps of each
// off-diagonal block pair (partner (l + s) mod G of block J > I).
#pragma once

#include <cstddef>

namespace amto {

// Float offset of (time block tb, global step sg, axis, warp lane, sample of
// the lane's pair tsel) in one instance's multiplier buffer, S4 = S / 4.
__host__ __device__ __forceinline__ size_t lam_index(int tb, int sg, int ax, int lane, int tsel,
                                                     int S4) {
    return ((size_t)(tb * S4 + (sg >> 2)) * 3 + ax) * 256 + tsel * 128 + lane * 4 + (sg & 3);
}

// Global step sg of a time block -> (block pair I, J, step s in the tile).
__device__ __forceinline__ void decode_step(int sg, int nbk, int G, int& I, int& J, int& s) {
    for (int i = 0; i < nbk; ++i) {
        if (sg < G / 2) { I = i; J = i; s = 1 + sg; return; }
        sg -= G / 2;
        int row = (nbk - 1 - i) * G;
        if (sg < row) { I = i; J = i + 1 + sg / G; s = sg % G; return; }
        sg -= row;
    }
    I = J = s = 0;
}

// Schedule position of the unordered pair (i < j) at sample t, and the sign
// of its stored multiplier (-1 when the schedule forms it as j - i).
__device__ __forceinline__ void pair_slot(int i, int j, int t, int G, int nbk, int& tb, int& sg,
                                          int& lane, int& tsel, float& sigma) {
    const int TB = 64 / G;
    const int I = i / G, J = j / G, li = i % G, lj = j % G;
    int off = 0, step, l;
    sigma = 1.f;
    for (int r = 0; r < I; ++r) off += G / 2 + (nbk - 1 - r) * G;
    if (I < J) {
        off += G / 2 + (J - I - 1) * G;
        step = (lj - li + G) % G;
        l = li;
    } else {
        const int d = lj - li;  // 1..G-1
        if (d <= G / 2) { step = d - 1; l = li; }
        else { step = G - d - 1; l = lj; sigma = -1.f; }
    }
    tb = t / TB;
    const int rr = t % TB;
    sg = off + step;
    lane = (rr / 2) * G + l;
    tsel = rr % 2;
}

}  // namespace amto
