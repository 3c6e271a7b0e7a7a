// ludax_hex_lanes.cuh -- Hex with several lanes cooperating on one env
// (threads_per_env = 2 or 4) for the single-game fused playouts.
//
// The board (n*n <= 121 cells, cell id = r*n + c as everywhere) is held as
// four 32-bit words, word i covering cells 32i .. 32i+31; the TPE lanes of a
// group each hold 4/TPE consecutive words of every bitboard (stones, the
// edge-connected sets of Sec. 4's incremental connectivity, the spreading
// front).  Work that is per word (legal cells, the neighbour dilation, the
// edge-set updates) is split across the lanes; the draw, the count of legal
// cells, the choice of the k-th one and the end tests are shared through
// warp shuffles and votes within the group.  A dilation moves bits across
// word boundaries, so each lane takes the last word of the lane before it
// and the first word of the lane after it (two shuffles per dilation).
//
// The rules, the draw keyed on (seed, global env, ply) and the spreading
// flood are those of Hex<N> (ludax_games.cuh): results are the same bit for
// bit; only the split of the work across lanes differs.
#pragma once
#include "ludax_games.cuh"

namespace ludax {

// word i (0..3) of a 128-bit Hex mask: kind 0 board, 1 column 0, 2 column
// n-1, 3 row 0, 4 row n-1
__host__ __device__ constexpr uint32_t hex_word32(int n, int i, int kind) {
    const uint64_t w = hex_word(n, i >> 1, kind);
    return (uint32_t)(w >> (32 * (i & 1)));
}

template <int N, int TPE>
struct HexLanes {
    static_assert(TPE == 2 || TPE == 4, "2 or 4 lanes per env");
    static constexpr int kCells = N * N, kCap = N * N, WPL = 4 / TPE;
    static constexpr int kGame = 3;

    uint32_t own[WPL], opp[WPL], ownA[WPL], ownB[WPL], oppA[WPL], oppB[WPL], front[WPL];
    // this lane's words of the constant masks, and of the masks of the word
    // just before / after its own (for bits that cross into its words)
    uint32_t board[WPL], col0[WPL], colL[WPL], row0[WPL], rowL[WPL];
    uint32_t ncl_prev, nc0_prev, ncl_next, nc0_next;  // board & ~column n-1 / ~column 0 of those words
    int side, ply, outcome;
    int r;           // rank of this lane in its group
    unsigned gmask;  // the group's lanes in the warp
    const uint32_t* nbr_table;  // [cells][4] neighbour words in shared memory, or nullptr

    __device__ __forceinline__ static uint32_t mask_at(int i, int kind) {
        // i is 0..3 or out of range (-1, 4): 0
        uint32_t m = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w) m = i == w ? hex_word32(N, w, kind) : m;
        return m;
    }
    __device__ __forceinline__ void init_lane(int rank, unsigned group_mask, const uint32_t* table) {
        r = rank;
        gmask = group_mask;
        nbr_table = table;
#pragma unroll
        for (int j = 0; j < WPL; ++j) {
            const int i = r * WPL + j;
            board[j] = mask_at(i, 0);
            col0[j] = mask_at(i, 1);
            colL[j] = mask_at(i, 2);
            row0[j] = mask_at(i, 3);
            rowL[j] = mask_at(i, 4);
        }
        const int ip = r * WPL - 1, in = r * WPL + WPL;
        ncl_prev = mask_at(ip, 0) & ~mask_at(ip, 2);
        nc0_prev = mask_at(ip, 0) & ~mask_at(ip, 1);
        ncl_next = mask_at(in, 0) & ~mask_at(in, 2);
        nc0_next = mask_at(in, 0) & ~mask_at(in, 1);
    }

    // ---- group-wide helpers (every lane of the group calls them together)
    __device__ __forceinline__ bool group_any(bool p) const { return __ballot_sync(gmask, p) != 0u; }
    // the six neighbours of the cells of s, on the board (the dilation of
    // Hex<N>::nbrs, word by word): shifts by n (row), 1 (column) and n-1 (the
    // anti-diagonal), with the column masks that stop wrap-around
    __device__ __forceinline__ void nbrs(const uint32_t (&s)[WPL], uint32_t (&out)[WPL]) const {
        uint32_t prev = __shfl_up_sync(gmask, s[WPL - 1], 1, TPE);
        uint32_t next = __shfl_down_sync(gmask, s[0], 1, TPE);
        if (r == 0) prev = 0u;
        if (r == TPE - 1) next = 0u;
        uint32_t e[WPL + 2], ea[WPL + 2], eb[WPL + 2];  // words i-1 .. i+WPL of s, s & ~col n-1, s & ~col 0
        e[0] = prev;
        ea[0] = prev & ncl_prev;
        eb[0] = prev & nc0_prev;
#pragma unroll
        for (int j = 0; j < WPL; ++j) {
            e[j + 1] = s[j];
            ea[j + 1] = s[j] & board[j] & ~colL[j];
            eb[j + 1] = s[j] & board[j] & ~col0[j];
        }
        e[WPL + 1] = next;
        ea[WPL + 1] = next & ncl_next;
        eb[WPL + 1] = next & nc0_next;
#pragma unroll
        for (int j = 0; j < WPL; ++j) {
            // toward higher ids by S: (w << S) | (word below >> (32 - S)); toward lower: the mirror
            const uint32_t dn = __funnelshift_l(e[j], e[j + 1], N);          // (r+1, c)
            const uint32_t up = __funnelshift_r(e[j + 1], e[j + 2], N);      // (r-1, c)
            const uint32_t rt = __funnelshift_l(ea[j], ea[j + 1], 1);        // (r, c+1)
            const uint32_t lf = __funnelshift_r(eb[j + 1], eb[j + 2], 1);    // (r, c-1)
            const uint32_t ur = __funnelshift_r(ea[j + 1], ea[j + 2], N - 1);  // (r-1, c+1)
            const uint32_t dl = __funnelshift_l(eb[j], eb[j + 1], N - 1);    // (r+1, c-1)
            out[j] = (dn | up | rt | lf | ur | dl) & board[j];
        }
    }

    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int j = 0; j < WPL; ++j) own[j] = opp[j] = ownA[j] = ownB[j] = oppA[j] = oppB[j] = front[j] = 0u;
        side = ply = 0;
        outcome = kOngoing;
    }
    // this lane's words of a 128-bit plane pair (lo, hi)
    __device__ __forceinline__ void words_of(uint64_t lo, uint64_t hi, uint32_t (&w)[WPL]) const {
#pragma unroll
        for (int j = 0; j < WPL; ++j) {
            const int i = r * WPL + j;
            const uint64_t q = i < 2 ? lo : hi;
            w[j] = (uint32_t)(q >> (32 * (i & 1)));
        }
    }
    // the 64-bit plane word k (0 = cells 0..63, 1 = cells 64..127) of v,
    // assembled from the group's lanes (every lane gets it)
    __device__ __forceinline__ uint64_t plane_word(const uint32_t (&v)[WPL], int k) const {
        uint32_t lo32 = 0, hi32 = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int holder = i / WPL, j = i % WPL;
            uint32_t mine = 0;
#pragma unroll
            for (int jj = 0; jj < WPL; ++jj) mine = jj == j ? v[jj] : mine;
            const uint32_t x = __shfl_sync(gmask, mine, holder, TPE);
            if (i == 2 * k) lo32 = x;
            if (i == 2 * k + 1) hi32 = x;
        }
        return (uint64_t)lo32 | ((uint64_t)hi32 << 32);
    }

    // One layer of the last mover's (now opp's) spreading group, as
    // Hex<N>::spread; true while it still grows.
    __device__ __forceinline__ bool spread() {
        uint32_t fa = 0;
#pragma unroll
        for (int j = 0; j < WPL; ++j) fa |= front[j] & oppA[j];
        const bool to_a = group_any(fa != 0u);
        uint32_t nb[WPL];
        nbrs(front, nb);
        bool grew = false;
#pragma unroll
        for (int j = 0; j < WPL; ++j) {
            const uint32_t nw = nb[j] & opp[j] & ~(oppA[j] | oppB[j]);
            oppA[j] |= to_a ? nw : 0u;
            oppB[j] |= to_a ? 0u : nw;
            front[j] = nw;
            grew |= nw != 0u;
        }
        return group_any(grew);
    }
    // placement of `cell` with the flood left to spread(), as Hex<N>::place_spread
    __device__ __forceinline__ void place_spread(int cell) {
        uint32_t x[WPL], nx[WPL];
#pragma unroll
        for (int j = 0; j < WPL; ++j) x[j] = (cell >> 5) == r * WPL + j ? 1u << (cell & 31) : 0u;
        if (nbr_table) {
#pragma unroll
            for (int j = 0; j < WPL; ++j) nx[j] = nbr_table[cell * 4 + r * WPL + j];
        } else {
            nbrs(x, nx);
        }
        uint32_t ta = 0, tb = 0;
#pragma unroll
        for (int j = 0; j < WPL; ++j) {
            const uint32_t ea = side == 0 ? row0[j] : col0[j], eb = side == 0 ? rowL[j] : colL[j];
            ta |= (x[j] & ea) | (nx[j] & ownA[j]);
            tb |= (x[j] & eb) | (nx[j] & ownB[j]);
        }
        const bool touch_a = group_any(ta != 0u), touch_b = group_any(tb != 0u);
#pragma unroll
        for (int j = 0; j < WPL; ++j) own[j] |= x[j];
        if (touch_a && touch_b) {
            outcome = side + 1;
        } else if (touch_a || touch_b) {
#pragma unroll
            for (int j = 0; j < WPL; ++j) {
                const uint32_t first = nx[j] & own[j] & ~(ownA[j] | ownB[j]);
                const uint32_t c = x[j] | first;
                ownA[j] |= touch_a ? c : 0u;
                ownB[j] |= touch_a ? 0u : c;
                front[j] = first;
            }
        }
        ++ply;
#pragma unroll
        for (int j = 0; j < WPL; ++j) {
            uint32_t t = own[j]; own[j] = opp[j]; opp[j] = t;
            t = ownA[j]; ownA[j] = oppA[j]; oppA[j] = t;
            t = ownB[j]; ownB[j] = oppB[j]; oppB[j] = t;
        }
        side ^= 1;
    }
    // one loop step: grow a spreading group, else play one uniform-random ply
    // (k-th legal cell in ascending id for k = umulhi(top 32 bits of the draw, count))
    __device__ __forceinline__ void step(uint64_t key, uint32_t& rhi) {
        if (spread()) return;
        const uint32_t rnext = draw_hi(key, (uint32_t)ply + 1u);
        uint32_t m[WPL];
        int c = 0;
#pragma unroll
        for (int j = 0; j < WPL; ++j) {
            m[j] = board[j] & ~(own[j] | opp[j]);
            c += __popc(m[j]);
        }
        int incl = c;
#pragma unroll
        for (int d = 1; d < TPE; d <<= 1) {
            const int t = __shfl_up_sync(gmask, incl, d, TPE);
            if (r >= d) incl += t;
        }
        const int total = __shfl_sync(gmask, incl, TPE - 1, TPE);
        const int k = (int)__umulhi(rhi, (uint32_t)total), excl = incl - c;
        const bool mine = k >= excl && k < incl;
        int cell = 0;
        if (mine) {
            int p;
            if constexpr (WPL == 1) p = select_bit(m[0], (uint32_t)(k - excl));
            else p = select_bit((uint64_t)m[0] | ((uint64_t)m[1] << 32), (uint32_t)(k - excl));
            cell = r * WPL * 32 + p;
        }
        const unsigned who = __ballot_sync(gmask, mine);
        cell = __shfl_sync(gmask, cell, __ffs(who) - 1);
        place_spread(cell);
        if (outcome == kOngoing && ply >= kCap) outcome = kCapped;
        rhi = rnext;
    }
    __device__ __forceinline__ void settle() {
#pragma unroll 1
        while (spread()) {
        }
    }
};

}  // namespace ludax
