// Size-specialised instantiations of the FFT-carrying kernels: candidate lists.
//
// Each macro appends one compile-time configuration for axis length N (the kernels and
// their grouped forms) to the candidate list `out` of the requested role (see
// kernel_candidates in eval.cuh);
// the first candidate of a role is its default, and the autotuner times the others
// at a grid's first evaluation.
//   OFDFT_CAND_ROW(T, N, RB, NT, MAXR, MINB)    per-channel row kernels: RB row pairs per
//                                               block (batch stride RB + 1), NT threads
//   OFDFT_CAND_ROW2(T, N, G, NT, MAXR, MINB)    channel-batched row kernels: one pair of rows
//                                               per block, G channels per transform
//   OFDFT_CAND_PENCIL(T, N, TW, NT, MAXR, MINB) n1 pencils: TW columns per tile
//   OFDFT_CAND_AXIS0(T, N, TW, NT, MAXR, MINB)  column-tile reciprocal-space kernel: TW columns
// MAXR caps the radix of the transform, MINB sets the minimum resident blocks per SM
// (0 = the policy's default).  Each thread stages at most ceil((N/R) * batch / NT)
// butterflies per pass.
#pragma once

#include <cstdio>

#include "kernels.cuh"

namespace ofdft {
inline KernelCand make_cand(const void *k1, const void *k2, const void *g1, const void *g2, int B, int nt,
                            const char *kind, int maxr, int minb) {
    KernelCand c;
    c.batched = kind[4] == '2';
    c.k1 = k1;
    c.k2 = k2;
    c.g1 = g1;
    c.g2 = g2;
    c.B = B;
    c.nt = nt;
    std::snprintf(c.name, sizeof(c.name), "%s %dx%d r%d b%d", kind, B, nt, maxr, minb);
    return c;
}
}  // namespace ofdft

#define OFDFT_CAND_ROW(T, N, RB, NT, MAXR, MINB)                                                        \
    if (role == ROLE_ROW && n == N) {                                                                   \
        typedef ::ofdft::CtPolicy<T, N, RB, RB + 1, NT, MAXR, MINB> PR;                                 \
        out.push_back(make_cand((const void *)row_fwd_kernel<T, PR>, (const void *)row_inv_kernel<T, PR>, \
                                (const void *)row_fwd_group<T, PR>, (const void *)row_inv_group<T, PR>,   \
                                RB, NT, "rows", MAXR, MINB));                                           \
    }

#define OFDFT_CAND_ROW2(T, N, G, NT, MAXR, MINB)                                                        \
    if (role == ROLE_ROW2 && n == N) {                                                                  \
        typedef ::ofdft::RowPolicy2<T, N, G, NT, MAXR, MINB> PQ;                                        \
        out.push_back(make_cand((const void *)row_fwd2_kernel<T, PQ>, (const void *)row_inv2_kernel<T, PQ>, \
                                (const void *)row_fwd2_group<T, PQ>, (const void *)row_inv2_group<T, PQ>, \
                                G, NT, "rows2", MAXR, MINB));                                           \
    }

#define OFDFT_CAND_PENCIL(T, N, TW, NT, MAXR, MINB)                                                     \
    if (role == ROLE_PENCIL && n == N) {                                                                \
        typedef ::ofdft::CtPolicy<T, N, TW, TW, NT, MAXR, MINB> PP;                                     \
        out.push_back(make_cand((const void *)pencil1_kernel<T, -1, PP>, (const void *)pencil1_kernel<T, +1, PP>, \
                                (const void *)pencil1_group<T, -1, PP>, (const void *)pencil1_group<T, +1, PP>, \
                                TW, NT, "pencil", MAXR, MINB));                                         \
    }

// (out of place or in place as axis0_oop<T>(N) says, which the host also uses for its scratch);
// k1 is the Wang-Teter form, k2 the Eq. MGP form
#define OFDFT_CAND_AXIS0(T, N, TW, NT, MAXR, MINB)                                                      \
    if (role == ROLE_AXIS0 && n == N) {                                                                 \
        typedef ::ofdft::CtPolicy<T, N, TW, TW, NT, MAXR, MINB, ::ofdft::axis0_oop<T>(N)> PA;           \
        out.push_back(make_cand((const void *)axis0_kernel<T, PA, false>, (const void *)axis0_kernel<T, PA, true>, \
                                (const void *)axis0_group<T, PA, false>, (const void *)axis0_group<T, PA, true>, \
                                TW, NT, "tile", MAXR, MINB));                                           \
    }

// the common set for one length: rows, pencils and the tile reciprocal-space kernel
#define OFDFT_CAND_ALL(T, N, RB, RNT, PTW, PNT, ATW, ANT)                                               \
    OFDFT_CAND_ROW(T, N, RB, RNT, (sizeof(T) == 4 ? 16 : 8), 0)                                         \
    OFDFT_CAND_PENCIL(T, N, PTW, PNT, (sizeof(T) == 4 ? 16 : 8), 0)                                     \
    OFDFT_CAND_AXIS0(T, N, ATW, ANT, (sizeof(T) == 4 ? 16 : 8), 0)
