// ludax_state.cuh -- env state in HBM (structure of arrays) and the
// persistent playout loop shared by the single-game and mixed-game kernels.
//
// HBM layout of an env batch of n envs (all arrays length n, coalesced by env):
//   planes[k*n + e]  uint64 bitboard planes in the game's internal layout
//                    TTT/C4/Reversi: k=0 P1 stones, k=1 P2 stones
//                    Hex: k=0,1 P1 stones (lo, hi word), k=2,3 P2 stones,
//                         k=4,5 P1 edge-A set, k=6,7 P1 edge-B set,
//                         k=8,9 P2 edge-A set, k=10,11 P2 edge-B set
//                    Gomoku/Pente/Yavalath: k = 0..W-1 P1 words, W..2W-1 P2 words
//                    Wolf and Sheep: P1, P2 pieces; Draughts: P1 men, P1
//                    kings, P2 men, P2 kings; Dai Hasami Shogi: P1 lo/hi, P2 lo/hi
//   meta[e]          uint32: bits 0-7 ply (low byte), 8-9 passes, 10 side to
//                    move (0 = P1), 12-14 outcome+1 (0 ongoing), 15 illegal
//                    flag, 16-23 ply (high byte), 24-27 / 28-31 pairs captured
//                    by P1 / P2 (Pente); 24-31 Draughts: 1 + the cell of the
//                    piece that must hop again (0 if none)
#pragma once
#include "ludax_games.cuh"

namespace ludax {

struct EnvDev {
    uint64_t* planes;
    uint32_t* meta;
    int64_t n;
    int64_t env_offset;
    unsigned long long* counters;  // [0] refill cursor, [1] illegal actions, [2] capped envs
    int32_t desc;                  // the env's game descriptor (parameters of the line game)
    int32_t cells;                 // cells per board in canonical views
};

__device__ __forceinline__ uint32_t pack_meta(int ply, int passes, int side, int outcome, int illegal, int caps1 = 0,
                                              int caps2 = 0) {
    return (uint32_t)(ply & 0xFF) | ((uint32_t)(passes & 3) << 8) | ((uint32_t)(side & 1) << 10) |
           ((uint32_t)((outcome + 1) & 7) << 12) | ((uint32_t)(illegal & 1) << 15) |
           ((uint32_t)((ply >> 8) & 0xFF) << 16) | ((uint32_t)(caps1 & 15) << 24) | ((uint32_t)(caps2 & 15) << 28);
}
__device__ __forceinline__ void unpack_meta(uint32_t m, int& ply, int& passes, int& side, int& outcome) {
    ply = (int)(m & 0xFF) | (int)(((m >> 16) & 0xFF) << 8);
    passes = (int)((m >> 8) & 3);
    side = (int)((m >> 10) & 1);
    outcome = (int)((m >> 12) & 7) - 1;
}

template <class G>
struct HexN {
    static constexpr int value = 0;
};
template <int N>
struct HexN<Hex<N>> {
    static constexpr int value = N;
};
// number of 64-bit words per player for the multi-word bitboard games
template <class G>
struct WideW {
    static constexpr int value = 0;
};
template <>
struct WideW<Gomoku> {
    static constexpr int value = Gomoku::W;
};
template <>
struct WideW<Pente> {
    static constexpr int value = Pente::W;
};
template <>
struct WideW<Yavalath> {
    static constexpr int value = Yavalath::W;
};
template <>
struct WideW<LineGame> {
    static constexpr int value = LineGame::W;
};

// -------------------------------------------------------- load / store --
template <class G>
__device__ __forceinline__ void load_state(G& g, const EnvDev& d, int64_t e) {
    configure(g, d.desc);
    const uint32_t meta = d.meta[e];
    unpack_meta(meta, g.ply, g.passes, g.side, g.outcome);
    if constexpr (IsMove<G>::value) {
        uint64_t w[G::kPlanes];
#pragma unroll
        for (int k = 0; k < G::kPlanes; ++k) w[k] = d.planes[(int64_t)k * d.n + e];
        g.planes_in(w);
        g.set_extra((int)((meta >> 24) & 0xFF));
    } else if constexpr (WideW<G>::value != 0) {
        constexpr int W = WideW<G>::value;
        typename G::Mask p1, p2;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            p1.w[i] = d.planes[(int64_t)i * d.n + e];
            p2.w[i] = d.planes[(int64_t)(W + i) * d.n + e];
        }
        g.own = g.side == 0 ? p1 : p2;
        g.opp = g.side == 0 ? p2 : p1;
        if constexpr (G::kGame == Pente::kGame) {
            const int c1 = (int)((meta >> 24) & 15), c2 = (int)((meta >> 28) & 15);
            g.caps_own = g.side == 0 ? c1 : c2;
            g.caps_opp = g.side == 0 ? c2 : c1;
        }
    } else if constexpr (HexN<G>::value == 0) {
        uint64_t p1 = d.planes[e], p2 = d.planes[d.n + e];
        uint64_t own = g.side == 0 ? p1 : p2, opp = g.side == 0 ? p2 : p1;
        g.own = (typename G::Mask)own;
        g.opp = (typename G::Mask)opp;
    } else {
        const uint64_t* P = d.planes;
        const int64_t n = d.n;
        B128 s1 = {P[0 * n + e], P[1 * n + e]}, s2 = {P[2 * n + e], P[3 * n + e]};
        B128 a1 = {P[4 * n + e], P[5 * n + e]}, b1 = {P[6 * n + e], P[7 * n + e]};
        B128 a2 = {P[8 * n + e], P[9 * n + e]}, b2 = {P[10 * n + e], P[11 * n + e]};
        bool p1 = g.side == 0;
        g.own = p1 ? s1 : s2;
        g.opp = p1 ? s2 : s1;
        g.ownA = p1 ? a1 : a2;
        g.ownB = p1 ? b1 : b2;
        g.oppA = p1 ? a2 : a1;
        g.oppB = p1 ? b2 : b1;
        g.front = B128{0, 0};  // a stored state is settled
    }
    refresh_of(g);
}

template <class G>
__device__ __forceinline__ void store_state(const G& g, const EnvDev& d, int64_t e, int illegal = 0) {
    if constexpr (IsMove<G>::value) {
        const int x = g.extra();
        d.meta[e] = pack_meta(g.ply, g.passes, g.side, g.outcome, illegal, x & 15, (x >> 4) & 15);
        uint64_t w[G::kPlanes];
        g.planes_out(w);
#pragma unroll
        for (int k = 0; k < G::kPlanes; ++k) d.planes[(int64_t)k * d.n + e] = w[k];
    } else if constexpr (WideW<G>::value != 0) {
        constexpr int W = WideW<G>::value;
        int c1 = 0, c2 = 0;
        if constexpr (G::kGame == Pente::kGame) {
            c1 = g.side == 0 ? g.caps_own : g.caps_opp;
            c2 = g.side == 0 ? g.caps_opp : g.caps_own;
        }
        d.meta[e] = pack_meta(g.ply, g.passes, g.side, g.outcome, illegal, c1, c2);
#pragma unroll
        for (int i = 0; i < W; ++i) {
            d.planes[(int64_t)i * d.n + e] = g.side == 0 ? g.own.w[i] : g.opp.w[i];
            d.planes[(int64_t)(W + i) * d.n + e] = g.side == 0 ? g.opp.w[i] : g.own.w[i];
        }
    } else if constexpr (HexN<G>::value == 0) {
        d.meta[e] = pack_meta(g.ply, g.passes, g.side, g.outcome, illegal);
        uint64_t own = (uint64_t)g.own, opp = (uint64_t)g.opp;
        d.planes[e] = g.side == 0 ? own : opp;
        d.planes[d.n + e] = g.side == 0 ? opp : own;
    } else {
        d.meta[e] = pack_meta(g.ply, g.passes, g.side, g.outcome, illegal);
        uint64_t* P = d.planes;
        const int64_t n = d.n;
        bool p1 = g.side == 0;
        B128 s1 = p1 ? g.own : g.opp, s2 = p1 ? g.opp : g.own;
        B128 a1 = p1 ? g.ownA : g.oppA, b1 = p1 ? g.ownB : g.oppB;
        B128 a2 = p1 ? g.oppA : g.ownA, b2 = p1 ? g.oppB : g.ownB;
        P[0 * n + e] = s1.lo; P[1 * n + e] = s1.hi;
        P[2 * n + e] = s2.lo; P[3 * n + e] = s2.hi;
        P[4 * n + e] = a1.lo; P[5 * n + e] = a1.hi;
        P[6 * n + e] = b1.lo; P[7 * n + e] = b1.hi;
        P[8 * n + e] = a2.lo; P[9 * n + e] = a2.hi;
        P[10 * n + e] = b2.lo; P[11 * n + e] = b2.hi;
    }
}

template <class G>
__device__ __forceinline__ void set_table(G& g, const B128* table) {
    if constexpr (HexN<G>::value != 0) g.nbr_table = table;
}

// is bit b of the internal mask set?
__device__ __forceinline__ bool mask_has(uint32_t m, int b) { return (m >> b) & 1u; }
__device__ __forceinline__ bool mask_has(uint64_t m, int b) { return (m >> b) & 1ull; }
__device__ __forceinline__ bool mask_has(B128 m, int b) { return b < 64 ? ((m.lo >> b) & 1ull) : ((m.hi >> (b - 64)) & 1ull); }
template <int W>
__device__ __forceinline__ bool mask_has(const BitsW<W>& m, int b) { return test_bit(m, b); }

// word w of a legal mask in canonical cell order
template <class G>
__device__ __forceinline__ uint64_t canon_mask_word(const G& g, const typename G::Mask& m, int w) {
    if constexpr (WideW<G>::value == 0) {
        return G::canon_word(m, w);
    } else {
        uint64_t out = 0;
        const int cells = cells_of(g);
        for (int j = 0; j < 64; ++j) {
            const int c = w * 64 + j;
            if (c < cells && mask_has(m, g.bit_of(c))) out |= 1ull << j;
        }
        return out;
    }
}

// ------------------------------------------------------------- refill --
// Warp-aggregated claim of one new work index per calling lane: the lanes
// that arrive together take consecutive indices with one atomic.
__device__ __forceinline__ long long claim_next(unsigned long long* cursor) {
    unsigned m = __activemask();
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(cursor, (unsigned long long)__popc(m));
    base = __shfl_sync(m, base, leader);
    return (long long)(base + __popc(m & ((1u << lane) - 1u)));
}

// cells holding a piece (any player)
template <class G>
__device__ __forceinline__ auto occupied_of(const G& g) {
    if constexpr (IsMove<G>::value) return g.occupied();
    else return g.own | g.opp;
}

// number of canonical actions (move games: from * cells + to)
template <class G>
__device__ __forceinline__ int actions_of(const G& g) {
    if constexpr (IsMove<G>::value) return G::kActions;
    else return cells_of(g) + (G::kHasPass ? 1 : 0);
}

// result of a finished game from P1's view: win 1, draw 0.5, loss 0
__device__ __forceinline__ float p1_score(int outcome) {
    return outcome == kWin1 ? 1.0f : (outcome == kWin2 ? 0.0f : 0.5f);
}

}  // namespace ludax
