// Size-specialised instantiations of the FFT-carrying kernels.
//
// OFDFT_SPECIALISE(T, N, RB, RNT, PTW, PNT, ATW, ANT) registers, for axis
// length N: the row kernels with RB row pairs per block (batch stride RB + 1)
// and RNT threads, the n1 pencil kernels with PTW columns and PNT threads, and
// the axis-0 kernel with ATW columns and ANT threads.  Each thread stages at
// most ceil((N/R) * batch / threads) butterflies per pass.
#pragma once

#include "kernels.cuh"

#define OFDFT_SPECIALISE(T, N, RB, RNT, PTW, PNT, ATW, ANT)                                   \
    OFDFT_SPECIALISE_X(T, N, RB, RNT, PTW, PNT, ATW, ANT, (sizeof(T) == 4 ? 16 : 8), (sizeof(T) == 4 ? 16 : 8), 0, 0)

// full form: RMAXR / AMAXR cap the radix of the row / axis-0 transforms, RMINB / AMINB
// override the minimum resident blocks of the row / axis-0 kernels (0 = default)
#define OFDFT_SPECIALISE_X(T, N, RB, RNT, PTW, PNT, ATW, ANT, RMAXR, AMAXR, RMINB, AMINB)        \
    if (n == N && role != ROLE_ROW2) {                                                        \
        typedef ::ofdft::CtPolicy<T, N, RB, RB + 1, RNT, RMAXR, RMINB> PR;                    \
        typedef ::ofdft::CtPolicy<T, N, PTW, PTW, PNT> PP;                                    \
        typedef ::ofdft::CtPolicy<T, N, ATW, ATW, ANT, AMAXR, AMINB, ::ofdft::axis0_oop<T>(N)> PA; \
        if (role == ROLE_ROW) {                                                               \
            *k1 = (const void *)row_fwd_kernel<T, PR>;                                        \
            *k2 = (const void *)row_inv_kernel<T, PR>;                                        \
            *B = RB;                                                                          \
            *nt = RNT;                                                                        \
        } else if (role == ROLE_PENCIL) {                                                     \
            *k1 = (const void *)pencil1_kernel<T, -1, PP>;                                    \
            *k2 = (const void *)pencil1_kernel<T, +1, PP>;                                    \
            *B = PTW;                                                                         \
            *nt = PNT;                                                                        \
        } else {                                                                              \
            *k1 = (const void *)axis0_kernel<T, PA, false>;                                   \
            *k2 = (const void *)axis0_kernel<T, PA, true>;                                    \
            *B = ATW;                                                                         \
            *nt = ANT;                                                                        \
        }                                                                                     \
        return true;                                                                          \
    }

// OFDFT_SPECIALISE_ROW2(T, N, G, NT, MAXR, MINB): the channel-batched row kernels
// for n2 = N (one pair of rows per block, G channels per transform, NT threads,
// at least MINB resident blocks per SM).
#define OFDFT_SPECIALISE_ROW2(T, N, G, NT, MAXR, MINB)                                        \
    if (role == ROLE_ROW2 && n == N) {                                                        \
        typedef ::ofdft::RowPolicy2<T, N, G, NT, MAXR, MINB> PQ;                              \
        *k1 = (const void *)row_fwd2_kernel<T, PQ>;                                           \
        *k2 = (const void *)row_inv2_kernel<T, PQ>;                                           \
        *B = G;                                                                               \
        *nt = NT;                                                                             \
        return true;                                                                          \
    }

// OFDFT_SPECIALISE_PENCIL(T, N, TW, NT, MINB): only the n1 pencil kernels for n1 = N, with at
// least MINB resident blocks per SM (tuning variants).
#define OFDFT_SPECIALISE_PENCIL(T, N, TW, NT, MINB)                                           \
    if (role == ROLE_PENCIL && n == N) {                                                      \
        typedef ::ofdft::CtPolicy<T, N, TW, TW, NT, (sizeof(T) == 4 ? 16 : 8), MINB> PP;      \
        *k1 = (const void *)pencil1_kernel<T, -1, PP>;                                        \
        *k2 = (const void *)pencil1_kernel<T, +1, PP>;                                        \
        *B = TW;                                                                              \
        *nt = NT;                                                                             \
        return true;                                                                          \
    }


// OFDFT_SPECIALISE_AXIS0(T, N, TW, NT, MAXR, MINB): only the reciprocal-space kernel for n0 = N
// (out of place or in place as axis0_oop<T>(N) says, which the host also uses for its scratch);
// k1 is the Wang-Teter form, k2 the Eq. MGP form.
#define OFDFT_SPECIALISE_AXIS0(T, N, TW, NT, MAXR, MINB)                                      \
    if (role == ROLE_AXIS0 && n == N) {                                                       \
        typedef ::ofdft::CtPolicy<T, N, TW, TW, NT, MAXR, MINB, ::ofdft::axis0_oop<T>(N)> PA;  \
        *k1 = (const void *)axis0_kernel<T, PA, false>;                                       \
        *k2 = (const void *)axis0_kernel<T, PA, true>;                                        \
        *B = TW;                                                                              \
        *nt = NT;                                                                             \
        return true;                                                                          \
    }
