// Reciprocal-space kernel with register-resident transforms along n0 and
// tensor-map (TMA) tile loads: the persistent form of the axis-0 pass of one
// evaluation (Sec. 2.3 s2 and the reciprocal half of s3, with the Hartree, local
// pseudopotential and von Weizsaecker products of Eq. efunc).
//
// Work unit: a tile of TW (even, at most 32) consecutive columns c = (k1, k2) of the half
// spectrum and all N values of k0.  MINB blocks per SM loop over the tiles t = b,
// b + (blocks), ...; a single thread keeps NSTAGE channel tiles in
// flight with cp.async.bulk.tensor copies (3-D tensor map over [channel][k0][c],
// one mbarrier per stage, bounded waits), across tile boundaries.
//
// Thread (w, t) = (threadIdx.x mod TW, threadIdx.x / TW) owns column w of the tile
// and, through every pass of the Stockham transform, the E = N / TC elements
// t + q TC + r N/R of that column (TC = number of column groups).  Each pass runs in registers; between passes
// the values go through a shared exchange tile (one barrier per exchange, two
// exchange tiles used alternately).  The forward transform ends with frequency
// k0 = t + q TC + r N/R_last in register q R_last + r, which is exactly the input
// order of the inverse transform with the radices reversed, so the reciprocal
// products are applied in registers and the inverse starts without an exchange.
// With TW = 32 a warp touches one row of 32 consecutive columns and with TW = 16 two
// rows of 16: every shared-memory access is conflict-free, and every global store
// whole 128- or 256-byte segments.  With TW = 14 or 28 (tiles that divide a 128 x 65
// column plane evenly over two rounds of the resident blocks) a warp spans parts of
// several tile rows: some exchange accesses take two wavefronts, and row segments start
// on 16-byte boundaries (the tensor copies' x coordinate stays a multiple of 16 bytes).
// rho^beta hat, the term-2 accumulator and |G| stay in registers for the whole tile.
#pragma once

#include <cuda.h>

#include "kernels.cuh"

namespace ofdft {
namespace rs {

// radices: greedily the largest of 16, 8, 4, 2, 5, 3 dividing both what is left of
// N and E (the per-thread element count), so that every pass gives each thread
// whole butterflies
constexpr int pick(int m, int E) {
    return (m % 16 == 0 && E % 16 == 0) ? 16
         : (m % 8 == 0 && E % 8 == 0)   ? 8
         : (m % 4 == 0 && E % 4 == 0)   ? 4
         : (m % 2 == 0 && E % 2 == 0)   ? 2
         : (m % 5 == 0 && E % 5 == 0)   ? 5
         : (m % 3 == 0 && E % 3 == 0)   ? 3
                                        : 0;
}
constexpr int npass(int N, int E) {
    int m = N, c = 0;
    while (m > 1) {
        const int r = pick(m, E);
        if (!r) return -1;
        m /= r;
        c++;
    }
    return c;
}
// radix of forward pass p
constexpr int radix(int N, int E, int p) {
    int m = N;
    for (int q = 0; q < p; q++) m /= pick(m, E);
    return pick(m, E);
}
// inverse pass p uses the forward radices in reverse order
constexpr int iradix(int N, int E, int p) { return radix(N, E, npass(N, E) - 1 - p); }
constexpr int fns(int N, int E, int p) {
    int s = 1;
    for (int q = 0; q < p; q++) s *= radix(N, E, q);
    return s;
}
constexpr int ins(int N, int E, int p) {
    int s = 1;
    for (int q = 0; q < p; q++) s *= iradix(N, E, q);
    return s;
}

// twiddles and butterflies of one pass on the thread's registers: butterfly q (of E/R) is
// j = t + q TC, its inputs in v[q R .. q R + R - 1]
template <int DIR, int N, int E, int TC, int R, int NS, typename C>
__device__ __forceinline__ void pass(C (&v)[E], int t, const C *tw) {
#pragma unroll
    for (int q = 0; q < E / R; q++) {
        if constexpr (NS > 1) {
            const int k = (t + q * TC) % NS;
#pragma unroll
            for (int r = 1; r < R; r++) {
                C w = tw[r * k * (N / (NS * R))];
                if (DIR > 0) w.y = -w.y;
                v[q * R + r] = cmul(v[q * R + r], w);
            }
        }
        dft<DIR, R>(&v[q * R]);
    }
}

// the outputs of a pass (radix R, NS) into the exchange tile X[e][TW]
template <int N, int E, int TC, int TW, int R, int NS, typename C>
__device__ __forceinline__ void put(const C (&v)[E], int t, int w, C *X) {
#pragma unroll
    for (int q = 0; q < E / R; q++) {
        const int j = t + q * TC, k = j % NS, base = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; r++) X[(base + r * NS) * TW + w] = v[q * R + r];
    }
}

// the inputs of a pass of radix R from a tile X[e][TW]: element j + r N/R of butterfly j
template <int N, int E, int TC, int TW, int R, typename C>
__device__ __forceinline__ void get(C (&v)[E], int t, int w, const C *X) {
#pragma unroll
    for (int q = 0; q < E / R; q++)
#pragma unroll
        for (int r = 0; r < R; r++) v[q * R + r] = X[(t + q * TC + r * (N / R)) * TW + w];
}

// passes p .. P-1 of a transform on the registers, with an exchange (put, block barrier,
// get) between consecutive passes; the exchange tiles alternate.  bar() returns true when
// a bounded wait failed, which ends the transform early (true is returned).
template <int DIR, int N, int E, int TC, int TW, int p, typename C, typename Bar>
__device__ __forceinline__ bool passes(C (&v)[E], int t, int w, const C *tw, C *Xa, C *Xb, bool &xsel, Bar &bar) {
    constexpr int P = npass(N, E);
    if constexpr (p < P) {
        constexpr int R = DIR < 0 ? radix(N, E, p) : iradix(N, E, p);
        constexpr int NS = DIR < 0 ? fns(N, E, p) : ins(N, E, p);
        pass<DIR, N, E, TC, R, NS>(v, t, tw);
        if constexpr (p + 1 < P) {
            C *X = xsel ? Xb : Xa;
            xsel = !xsel;
            put<N, E, TC, TW, R, NS>(v, t, w, X);
            if (bar()) return true;
            get<N, E, TC, TW, (DIR < 0 ? radix(N, E, p + 1) : iradix(N, E, p + 1))>(v, t, w, X);
        }
        return passes<DIR, N, E, TC, TW, p + 1>(v, t, w, tw, Xa, Xb, xsel, bar);
    } else {
        return false;
    }
}

}  // namespace rs

// ---------------------------------------------------------------- tensor copies
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Kernel parameters beside EvalArgs: the tensor maps of the channel workspace
// ([channel][k0][c] of T words) and of V_ext(G) (a one-channel map of the same shape).
struct RecipMaps {
    CUtensorMap chan;
    CUtensorMap vext;
};

template <typename T, int N, int E, int NSTAGE, int TW = 32> struct RecipShape {
    typedef typename Vec2<T>::type C;
    static constexpr int TC = N / E, NT = TW * TC, TILE = N * TW;
    static constexpr int BOXR = N > 256 ? 256 : N;    // rows per tensor copy (box limit 256)
    static constexpr size_t smem = (size_t)(NSTAGE + 2) * TILE * sizeof(C) + (size_t)N * sizeof(C) + 1024;
    static_assert(rs::npass(N, E) >= 2, "at least two passes");
    static_assert(N % BOXR == 0, "row boxes");
};

// Operations of one tile, in order (each one a channel of the workspace): the forward
// transform of the next loaded tile (fwd), the reciprocal-space product of the kind, and
// the inverse transform stored into channel `store` (< 0: nothing stored).
enum { OP_HPP = 0, OP_VW, OP_RB, OP_WT, OP_RR, OP_EX, OP_IP, OP_A };
struct RecipOp {
    signed char kind, fwd;
    short store, m;
};

template <typename T, int N, int E, int NSTAGE, bool MGP, int TW>
__device__ __forceinline__ void recip_body(const EvalArgs<T> &a, const RecipMaps &maps, const int bid,
                                           const int nblk) {
    typedef typename Vec2<T>::type C;
    typedef RecipShape<T, N, E, NSTAGE, TW> S;
    constexpr int TC = S::TC, NT = S::NT, TILE = S::TILE, P = rs::npass(N, E);
    constexpr int RL = rs::radix(N, E, P - 1);           // last forward radix
    constexpr int WPC = (int)(sizeof(C) / sizeof(T));    // T words per complex (2)
    // dynamic shared memory, rounded up to a 1 KB boundary (tensor-copy destinations are
    // 128-byte aligned; the launch adds 1 KB)
    extern __shared__ __align__(16) unsigned char recip_smem[];
    C *const stage = (C *)(recip_smem + ((1024u - (smem_u32(recip_smem) & 1023u)) & 1023u));
    C *const Xa = stage + NSTAGE * TILE;
    C *const Xb = Xa + TILE;
    C *const tw = Xb + TILE;
    __shared__ __align__(8) uint64_t full[NSTAGE];
    __shared__ int s_nload, s_nops;
    __shared__ double sd[4 * 32];
    __shared__ T sk[OFDFT_MAX_KNOTS];
    __shared__ int order[kMaxChan + 1];         // HPP, V_ext, vW, rho^beta, M knots: at most 4 + 64
    __shared__ RecipOp ops[kMaxChan + 2];
    // thread (w, t): column w of the tile, element set t (TW = 32: a warp is one t; TW = 16:
    // two t per warp, each half-warp one 128-byte row of every shared tile)
    const int w = threadIdx.x % TW, t = threadIdx.x / TW;
    const int n2h = a.n2h;
    const long long PL = (long long)a.n1 * n2h;
    const int ntile = (int)((PL + TW - 1) / TW);
    const bool lwt = a.kernel == 0, exact = a.nlpot == 0;
    const bool hp = a.terms & (8u | 16u), pp = a.terms & 16u;

    if (threadIdx.x == 0) {
        // loads of one tile in consumption order (channel slots; -1: V_ext(G)) and the operations
        int nl = 0, no = 0;
        auto op = [&](int kind, int fwd, int store, int m) {
            ops[no].kind = (signed char)kind;
            ops[no].fwd = (signed char)fwd;
            ops[no].store = (short)store;
            ops[no].m = (short)m;
            no++;
        };
        if (hp) {
            order[nl++] = CH_HPP;
            if (pp) order[nl++] = -1;
            op(OP_HPP, 1, CH_HPP, 0);
        }
        if (a.terms & 2u) {
            order[nl++] = CH_VW;
            op(OP_VW, 1, CH_VW, 0);
        }
        if (a.terms & 4u) {
            order[nl++] = CH_NL;
            op(OP_RB, 1, -1, 0);
            if (!lwt) {
                order[nl++] = CH_KNOT0;
                op(OP_WT, 1, CH_KNOT0, 0);
                op(OP_RR, 0, CH_NL, 0);
            } else {
                for (int m = 0; m < a.M; m++) {
                    if (exact) order[nl++] = CH_KNOT0 + m;
                    op(exact ? OP_EX : OP_IP, exact ? 1 : 0, CH_KNOT0 + m, m);
                }
                if (exact) op(OP_A, 0, CH_NL, 0);
            }
        }
        s_nload = nl;
        s_nops = no;
        for (int s = 0; s < NSTAGE; s++) mbar_init(&full[s], 1);
        fence_proxy_async_smem();
    }
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw0[i];
    if ((a.terms & 4u) && lwt)
        for (int i = threadIdx.x; i < a.M; i += NT) sk[i] = a.knots_t[i];
    __syncthreads();
    const int nload = s_nload, nops = s_nops;
    const int my_tiles = bid < ntile ? (ntile - 1 - bid) / nblk + 1 : 0;
    // (32-bit counters: at most (n1 (n2/2+1) / TW + 1) tiles of at most kMaxChan + 1 loads)
    const int total = my_tiles * nload;
    int issued = 0, cons = 0, pend = 0, L = 0;          // loads issued, released, read since the last barrier, next
    // thread 0: start loads while their stages are free
    auto refill = [&]() {
        if (threadIdx.x != 0) return;
        bool fenced = false;
        while (issued < total && issued < cons + NSTAGE) {
            const int ti = issued / nload, i = issued - ti * nload;
            const int c0 = (bid + ti * nblk) * TW;
            const int st = issued % NSTAGE;
            if (!fenced) {
                fence_proxy_async_smem();           // the stage was last read through the generic proxy
                fenced = true;
            }
            mbar_arrive_expect_tx(&full[st], (unsigned)(TILE * sizeof(C)));
            const int ch = order[i];
#pragma unroll
            for (int rb = 0; rb < N / S::BOXR; rb++) {
                C *dst = stage + st * TILE + rb * S::BOXR * TW;
                if (ch >= 0) tma_load_3d(dst, &maps.chan, c0 * WPC, rb * S::BOXR, ch, &full[st]);
                else tma_load_3d(dst, &maps.vext, c0 * WPC, rb * S::BOXR, 0, &full[st]);
            }
            issued++;
        }
    };
    // block barrier: true (in every thread alike) if a bounded wait of any thread failed
    // before it; otherwise what was read before it is released and its stages refilled.
    // After a failure nothing more is issued, and the loads from cons to issued are the
    // ones that may still be in flight.
    int wfail = 0;
    auto bar = [&]() -> bool {
        if (__syncthreads_or(wfail)) return true;
        cons += pend;
        pend = 0;
        refill();
        return false;
    };
    // the tile of load L (waits for it with a bounded number of polls)
    auto wait_load = [&]() -> const C * {
        const int st = L % NSTAGE;
        if (!mbar_wait_bounded(&full[st], (unsigned)((L / NSTAGE) & 1), a.wait_polls)) wfail = 1;
        L++;
        pend++;
        return stage + st * TILE;
    };
    refill();

    const T invN = (T)(1.0 / (double)a.N);
    double eH = 0.0, eV = 0.0, eP = 0.0, eN = 0.0;
    bool failed = false;
    C v[E], Rr[E], A[E];
    bool xsel = false;                         // exchange tile of the next exchange
    for (int ti = 0; ti < my_tiles && !failed; ti++) {
        const int col = (bid + ti * nblk) * TW + w;          // (n1 (n2/2+1) < 2^31)
        // this thread's column: its G components, half-spectrum weight, and |G| at its frequencies
        T cw, gn[E];
        {
            const int k1 = col / n2h, k2 = col - k1 * n2h;
            const double m1 = (k1 <= a.n1 / 2) ? k1 : k1 - a.n1, m2 = k2;
            T cv[3];
            for (int d = 0; d < 3; d++) cv[d] = (T)(m1 * a.bvec[3 + d] + m2 * a.bvec[6 + d]);
            cw = (col < PL) ? ((k2 == 0 || (a.n2 % 2 == 0 && k2 == a.n2 / 2)) ? (T)1 : (T)2) : (T)0;
#pragma unroll
            for (int q = 0; q < E / RL; q++)
#pragma unroll
                for (int r = 0; r < RL; r++) {
                    const int k0 = t + q * TC + r * (N / RL);
                    const T m0 = (T)(k0 <= N / 2 ? k0 : k0 - N);
                    const T gx = cv[0] + m0 * (T)a.bvec[0], gy = cv[1] + m0 * (T)a.bvec[1],
                            gz = cv[2] + m0 * (T)a.bvec[2];
                    gn[q * RL + r] = dsqrt(gx * gx + gy * gy + gz * gz);
                }
        }
        T gmin = gn[0];                                      // the smallest |G| of the thread
#pragma unroll
        for (int i = 1; i < E; i++) gmin = gn[i] < gmin ? gn[i] : gmin;
#pragma unroll
        for (int i = 0; i < E; i++) A[i] = cmake<C>((T)0, (T)0);
        for (int o = 0; o < nops; o++) {
            const RecipOp op = ops[o];
            if (op.fwd) {
                // forward transform of the next loaded tile: v in the last pass's frequency order
                rs::get<N, E, TC, TW, rs::radix(N, E, 0)>(v, t, w, wait_load());
                if ((failed = rs::passes<-1, N, E, TC, TW, 0>(v, t, w, tw, Xa, Xb, xsel, bar))) break;
            }
            const int kind = op.kind;
            if (kind == OP_WT || kind == OP_EX || kind == OP_IP) {
                // the kernel of this knot (WT: of the mean density's kF) at the thread's |G|
                const T hk = kind == OP_WT ? (T)(0.5 / a.scal[S_KF_WT]) : (T)0.5 / sk[op.m];
                Part<T, false> fN;
                // (a warp whose every eta is above 2 takes the kernel from the large-eta
                // polynomial alone: the same values, fewer instructions)
                auto knot = [&](auto large) {
#pragma unroll
                for (int i = 0; i < E; i++) {
                    T K;
                    if constexpr (decltype(large)::value) K = kernel_value_large(gn[i] * hk);
                    else K = kernel_value<T, MGP>(a, gn[i] * hk);
                    if (kind == OP_EX) {
                        // E_NL += Omega sum_G w Re(conj(FFT[h_m rho^alpha]) K_m FFT[rho^beta])
                        const C Sm = cscale(v[i], invN);
                        fN.add(cw * K * (Sm.x * Rr[i].x + Sm.y * Rr[i].y));
                        A[i] = cadd(A[i], cscale(Sm, K));
                        v[i] = cscale(Rr[i], K);
                    } else if (kind == OP_IP) {
                        v[i] = cscale(Rr[i], K);
                    } else {
                        // global-kF Wang-Teter: K rho^alpha hat to the knot channel, K rho^beta hat
                        // (kept for the next operation) to the rho^beta channel
                        const C Sa = cscale(v[i], invN);
                        fN.add(cw * K * (Sa.x * Rr[i].x + Sa.y * Rr[i].y));
                        Rr[i] = cscale(Rr[i], K);
                        v[i] = cscale(Sa, K);
                    }
                }
                };
                if (warp_all_large<T, MGP>(gmin, hk)) knot(std::true_type{});
                else knot(std::false_type{});
                eN += fN.value();
            } else if (kind == OP_HPP) {
                if (a.rhohat_out && col < PL) {
                    // the normalised density spectrum for the forces
#pragma unroll
                    for (int q = 0; q < E / RL; q++)
#pragma unroll
                        for (int r = 0; r < RL; r++)
                            a.rhohat_out[(size_t)(t + q * TC + r * (N / RL)) * PL + col] = cscale(v[q * RL + r], invN);
                }
                // Hartree + local pseudopotential (V_ext(G) tile at the thread's frequencies)
                C vx[E];
                if (pp) {
                    const C *X = wait_load();
#pragma unroll
                    for (int q = 0; q < E / RL; q++)
#pragma unroll
                        for (int r = 0; r < RL; r++) vx[q * RL + r] = X[(t + q * TC + r * (N / RL)) * TW + w];
                }
                Part<T, false> fH, fP;
#pragma unroll
                for (int i = 0; i < E; i++) {
                    const C X0 = cscale(v[i], invN);
                    const T g2 = gn[i] * gn[i];
                    C out = cmake<C>((T)0, (T)0);
                    if (g2 > (T)0) {
                        if (a.terms & 8u) {
                            const T f = (T)1 / g2;
                            fH.add(cw * (X0.x * X0.x + X0.y * X0.y) * f);
                            out = cscale(X0, (T)(4.0 * kPi) * f);
                        }
                        if (pp) {
                            fP.add(cw * (X0.x * vx[i].x + X0.y * vx[i].y));
                            out = cadd(out, vx[i]);
                        }
                    } else if (pp) {
                        out = vx[i];                      // G = 0: V_ext(0) only
                    }
                    v[i] = out;
                }
                eH += fH.value();
                eP += fP.value();
            } else if (kind == OP_VW) {
                // von Weizsaecker, psi form
                Part<T, false> fV;
#pragma unroll
                for (int i = 0; i < E; i++) {
                    const C X0 = cscale(v[i], invN);
                    const T g2 = gn[i] * gn[i];
                    fV.add(cw * g2 * (X0.x * X0.x + X0.y * X0.y));
                    v[i] = cscale(X0, g2);
                }
                eV += fV.value();
            } else if (kind == OP_RB) {
#pragma unroll
                for (int i = 0; i < E; i++) Rr[i] = cscale(v[i], invN);
            } else if (kind == OP_RR) {
#pragma unroll
                for (int i = 0; i < E; i++) v[i] = Rr[i];
            } else if (kind == OP_A) {
#pragma unroll
                for (int i = 0; i < E; i++) v[i] = A[i];
            }
            if (op.store >= 0) {
                // inverse transform and store of the column into the channel
                if ((failed = rs::passes<+1, N, E, TC, TW, 0>(v, t, w, tw, Xa, Xb, xsel, bar))) break;
                if (col < PL) {
                    constexpr int R1 = rs::radix(N, E, 0);
                    C *dst = a.chan + (size_t)op.store * a.NH + col;
#pragma unroll
                    for (int q = 0; q < E / R1; q++)
#pragma unroll
                        for (int r = 0; r < R1; r++) dst[(size_t)(t + q * TC + r * (N / R1)) * PL] = v[q * R1 + r];
                }
            }
        }
    }
    if (failed) {
        // a bounded wait expired: let every copy issued so far land (they target this
        // block's shared memory) with a longer bounded wait, count it and leave
        if (threadIdx.x == 0) {
            bool drained = true;
            for (int l = cons; l < issued; l++)
                drained = mbar_wait_bounded(&full[l % NSTAGE], (unsigned)((l / NSTAGE) & 1), 1u << 26) && drained;
            atomicAdd(a.scal + (drained ? S_TIMEOUT : S_FATAL), 1.0);
        }
        return;
    }
    double r4[4] = {eH, eV, eP, eN};
    block_sum_n<4>(r4, sd);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; k++) a.part_ax0[4 * bid + k] = r4[k];
}

// single evaluation (tensor maps in the parameter space)
template <typename T, int N, int E, int NSTAGE, bool MGP, int TW = 32, int MINB = 1>
__global__ void __launch_bounds__(TW * (N / E), MINB)
    recip_kernel(const EvalArgs<T> a, const __grid_constant__ RecipMaps maps) {
    recip_body<T, N, E, NSTAGE, MGP, TW>(a, maps, blockIdx.x, gridDim.x);
}

// grouped (see the grouped wrappers of kernels.cuh): evaluation k's arguments at ga[k], its
// tensor maps at maps.m[k] (parameter space, at most kGroupMax evaluations per launch)
struct RecipMapsGroup {
    RecipMaps m[kGroupMax];
};
template <typename T, int N, int E, int NSTAGE, bool MGP, int TW = 32, int MINB = 1>
__global__ void __launch_bounds__(TW * (N / E), MINB)
    recip_group(const EvalArgs<T> *__restrict__ ga, int bps, const __grid_constant__ RecipMapsGroup maps) {
    OFDFT_GROUP_INDEX;
    recip_body<T, N, E, NSTAGE, MGP, TW>(ga[gk], maps.m[gk], gb, bps);
}

}  // namespace ofdft
