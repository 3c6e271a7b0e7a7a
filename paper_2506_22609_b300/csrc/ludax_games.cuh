// ludax_games.cuh -- per-game bitboard code for the B300 engine (device side).
//
// Each game is a small struct whose whole state lives in registers:
//   own/opp   stones of the player to move and of the other player
//   side      0 when P1 is to move, 1 when P2 is
//   ply       plies played (passes included), passes (Reversi), outcome
// and whose methods implement the rules of the paper's game appendix (App. C)
// with the action = destination-cell convention (Sec. 3.4):
//   legal()   the legal-destination mask in the game's internal bit layout
//   place(b)  put a stone on internal bit b, apply effects and end rules
//   pass()    the forced pass (Reversi only, force_pass of App. B)
// The internal bit order of every layout is monotone in the canonical cell id
// (row-major, row 0 at the top), so "the k-th set bit" of a legal mask is the
// k-th legal cell in ascending canonical id.
//
// Layouts:
//   Tic-Tac-Toe  9 bits, bit = cell id; 8 line masks (the precomputed line
//                indices of Sec. 4, as bitmasks)
//   Connect Four 6 rows x 8-bit stride (column 7 always empty), bit = r*8+c;
//                the empty padding column stops shifted lines from wrapping,
//                so a line of four is b & b>>s & b>>2s & b>>3s for s in
//                {1 (row), 8 (column), 7 and 9 (diagonals)}; gravity: a cell
//                is legal when empty and the cell below (bit+8) is occupied
//                or it is on the bottom row
//   Reversi      8x8, bit = cell id; legal moves and flips by Kogge-Stone
//                occluded fills in 8 directions, with the opponent mask
//                restricted to columns 1..6 for every direction with a
//                horizontal component (no wrap across rows)
//   Hex n x n    n*n <= 121 bits in two 64-bit words, bit = cell id; six
//                neighbours (r-1,c) (r+1,c) (r,c-1) (r,c+1) (r-1,c+1)
//                (r+1,c-1) by shifts n, 1, n-1 with column masks.  Win
//                detection keeps, per player, the stones connected to each
//                of its two edges (A, B): a new stone joins edge A when it
//                lies on edge A or touches a stone of A, likewise for B; the
//                player wins when the stone joins both.  When it joins one,
//                the stones not yet connected to any edge that it links are
//                added to that set by a flood fill.  This is the incremental
//                connected-component update of Sec. 4 ("Dynamic State
//                Attributes") in bitboard form.  The fused playouts spread
//                that flood one layer per loop step instead (place_spread /
//                spread): every lane runs the same one-layer dilation each
//                step, and an env plays its next ply only once its flood has
//                stopped, so the lanes of a warp no longer wait for the
//                longest flood of the warp at every ply.
//   Gomoku 15x15 / Pente 19x19 / Yavalath: W-word bitboards (BitsW) with one
//                empty padding column per row (strides 16, 20 and 10), so
//                shifted line and capture patterns cannot wrap across rows;
//                Yavalath's 61-cell hexagon sits in axial coordinates (row r,
//                column c, |r - c| <= 4) of a 9x9 grid.
#pragma once
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace ludax {

constexpr int kOngoing = -1, kDraw = 0, kWin1 = 1, kWin2 = 2, kCapped = 3;

// ----------------------------------------------------------------- RNG --
// splitmix64 output function (Steele, Lea & Flood 2014): golden-ratio
// increment then the 30/27/31 xor-shift-multiply finaliser.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// key of a global env index given sm(seed)
__device__ __forceinline__ uint64_t env_key(uint64_t seed_key, uint64_t env) { return splitmix64(seed_key ^ env); }
// uniform index in [0, n) for this ply: top 32 bits of the draw times n, high word
__device__ __forceinline__ uint32_t draw_index(uint64_t key, uint32_t ply, uint32_t n) {
    uint64_t r = splitmix64(key ^ (uint64_t)ply);
    return __umulhi((uint32_t)(r >> 32), n);
}

// ---------------------------------------------------------- bit helpers --
struct B128 {
    uint64_t lo, hi;
};
__host__ __device__ __forceinline__ B128 operator|(B128 a, B128 b) { return {a.lo | b.lo, a.hi | b.hi}; }
// a | b for a and b with no bit in common, computed as adds (no carry can
// arise): an add also issues to a second pipe, where the logic ops the
// bitboard code is bound by have one
__host__ __device__ __forceinline__ B128 add_disjoint(B128 a, B128 b) { return {a.lo + b.lo, a.hi + b.hi}; }
__host__ __device__ __forceinline__ B128 operator&(B128 a, B128 b) { return {a.lo & b.lo, a.hi & b.hi}; }
__host__ __device__ __forceinline__ B128 operator~(B128 a) { return {~a.lo, ~a.hi}; }
__host__ __device__ __forceinline__ bool operator==(B128 a, B128 b) { return a.lo == b.lo && a.hi == b.hi; }
__host__ __device__ __forceinline__ bool any(B128 a) { return (a.lo | a.hi) != 0; }
__host__ __device__ __forceinline__ bool any(uint64_t a) { return a != 0; }
__host__ __device__ __forceinline__ bool any(uint32_t a) { return a != 0; }
template <int S>
__device__ __forceinline__ B128 shl(B128 a) {  // 0 < S < 64
    return {a.lo << S, (a.hi << S) | (a.lo >> (64 - S))};
}
template <int S>
__device__ __forceinline__ B128 shr(B128 a) {
    return {(a.lo >> S) | (a.hi << (64 - S)), a.hi >> S};
}
__device__ __forceinline__ B128 bit128(int b) {
    return {b < 64 ? (1ull << b) : 0ull, b >= 64 ? (1ull << (b - 64)) : 0ull};
}

__device__ __forceinline__ uint32_t popc(uint32_t m) { return __popc(m); }
__device__ __forceinline__ uint32_t popc(uint64_t m) { return __popcll(m); }
__device__ __forceinline__ uint32_t popc(B128 m) { return __popcll(m.lo) + __popcll(m.hi); }

// Position of the k-th set bit (k < popc(w)), branch-free and without
// popcount instructions on the dependent path (popcount and count-leading-
// zeros take ~19 cycles on sm_103a against ~5 for logic ops).  Nested SWAR
// counts give every 2-, 4- and 8-bit field's population at once; one
// multiply turns the byte counts into inclusive byte prefix sums; the byte
// holding the bit is found with three independent compares, then two
// field-halving steps and the last bit finish the search.
struct Swar32 {
    uint32_t w, a, b, p;  // word; 2-bit counts; 4-bit counts; byte prefix sums
};
__device__ __forceinline__ Swar32 swar32(uint32_t w) {
    Swar32 s;
    s.w = w;
    s.a = w - ((w >> 1) & 0x55555555u);
    s.b = (s.a & 0x33333333u) + ((s.a >> 2) & 0x33333333u);
    s.p = ((s.b + (s.b >> 4)) & 0x0F0F0F0Fu) * 0x01010101u;
    return s;
}
__device__ __forceinline__ uint32_t swar_select(const Swar32& s, uint32_t k) {
    const uint32_t p0 = s.p & 0xFFu, p1 = (s.p >> 8) & 0xFFu, p2 = (s.p >> 16) & 0xFFu;
    const uint32_t g0 = k >= p0, g1 = k >= p1, g2 = k >= p2;
    const uint32_t before = g2 ? p2 : (g1 ? p1 : (g0 ? p0 : 0u));
    uint32_t pos = (g0 + g1 + g2) << 3;
    k -= before;
    uint32_t c = (s.b >> pos) & 0xFu, t = k >= c;
    k -= t ? c : 0u;
    pos += t << 2;
    c = (s.a >> pos) & 3u;
    t = k >= c;
    k -= t ? c : 0u;
    pos += t << 1;
    c = (s.w >> pos) & 1u;
    return pos + (k >= c ? 1u : 0u);
}
__device__ __forceinline__ int select_bit(uint32_t m, uint32_t k) { return (int)swar_select(swar32(m), k); }
// the half that holds the k-th bit is chosen by the low half's count, then
// one SWAR search runs in it
__device__ __forceinline__ int select_bit(uint64_t m, uint32_t k) {
    const uint32_t lo = (uint32_t)m, hi = (uint32_t)(m >> 32);
    const uint32_t nlo = __popc(lo);
    const bool low = k < nlo;
    return (int)((low ? 0u : 32u) + swar_select(swar32(low ? lo : hi), low ? k : k - nlo));
}
__device__ __forceinline__ int select_bit(B128 m, uint32_t k) {
    const uint32_t c = __popcll(m.lo);
    const bool low = k < c;
    return (low ? 0 : 64) + select_bit(low ? m.lo : m.hi, low ? k : k - c);
}

// per-env scalars packed into one word for the shared-memory slot of an env
__device__ __forceinline__ uint64_t pack_small(int ply, int passes, int side, int outcome) {
    return (uint64_t)(ply & 0xFFFF) | ((uint64_t)(passes & 0xFF) << 16) | ((uint64_t)(side & 1) << 24) |
           ((uint64_t)(outcome + 1) << 32);
}
__device__ __forceinline__ void unpack_small(uint64_t w, int& ply, int& passes, int& side, int& outcome) {
    ply = (int)(w & 0xFFFF);
    passes = (int)((w >> 16) & 0xFF);
    side = (int)((w >> 24) & 1);
    outcome = (int)(w >> 32) - 1;
}

// ----------------------------------------------------------- Tic-Tac-Toe --
struct TTT {
    static constexpr int kGame = 0, kRows = 3, kCols = 3, kCells = 9, kCap = 9, kPlanes = 2;
    static constexpr bool kHasPass = false;
    using Mask = uint32_t;
    uint32_t own, opp;
    int side, ply, passes, outcome;

    __device__ __forceinline__ void reset() {
        own = opp = 0;
        side = ply = passes = 0;
        outcome = kOngoing;
    }
    __device__ __forceinline__ Mask legal() const { return ~(own | opp) & 0x1FFu; }
    __device__ __forceinline__ static bool line3(uint32_t b) {
        return ((b & 0x007u) == 0x007u) | ((b & 0x038u) == 0x038u) | ((b & 0x1C0u) == 0x1C0u) |
               ((b & 0x049u) == 0x049u) | ((b & 0x092u) == 0x092u) | ((b & 0x124u) == 0x124u) |
               ((b & 0x111u) == 0x111u) | ((b & 0x054u) == 0x054u);
    }
    __device__ __forceinline__ void place(int b) {
        own |= 1u << b;
        if (line3(own)) outcome = side + 1;
        else if ((own | opp) == 0x1FFu) outcome = kDraw;
        ++ply;
        uint32_t t = own; own = opp; opp = t;
        side ^= 1;
    }
    __device__ __forceinline__ void pass() {}
    __device__ __forceinline__ static int canon_of(int b) { return b; }
    __device__ __forceinline__ static int bit_of(int cell) { return cell; }
    __device__ __forceinline__ static uint64_t canon_word(Mask m, int w) { return w == 0 ? (uint64_t)m : 0ull; }
    // register state as kWords 64-bit words (shared-memory slots)
    static constexpr int kWords = 2;
    __device__ __forceinline__ void save(uint64_t* w) const {
        w[0] = (uint64_t)own | ((uint64_t)opp << 32);
        w[1] = pack_small(ply, passes, side, outcome);
    }
    __device__ __forceinline__ void load(const uint64_t* w) {
        own = (uint32_t)w[0];
        opp = (uint32_t)(w[0] >> 32);
        unpack_small(w[1], ply, passes, side, outcome);
    }
};

// ---------------------------------------------------------- Connect Four --
struct C4 {
    static constexpr int kGame = 1, kRows = 6, kCols = 7, kCells = 42, kCap = 42, kPlanes = 2;
    static constexpr bool kHasPass = false;
    static constexpr uint64_t kValid = 0x7F7F7F7F7F7Full;   // rows 0..5, columns 0..6
    static constexpr uint64_t kBottom = 0x7Full << 40;       // row 5
    using Mask = uint64_t;
    uint64_t own, opp;
    int side, ply, passes, outcome;

    __device__ __forceinline__ void reset() {
        own = opp = 0;
        side = ply = passes = 0;
        outcome = kOngoing;
    }
    __device__ __forceinline__ Mask legal() const {
        uint64_t occ = own | opp;
        return kValid & ~occ & ((occ >> 8) | kBottom);
    }
    __device__ __forceinline__ static bool line4(uint64_t b) {
        uint64_t h = b & (b >> 1), v = b & (b >> 8), d1 = b & (b >> 7), d2 = b & (b >> 9);
        return ((h & (h >> 2)) | (v & (v >> 16)) | (d1 & (d1 >> 14)) | (d2 & (d2 >> 18))) != 0;
    }
    __device__ __forceinline__ void place(int b) {
        own |= 1ull << b;
        if (line4(own)) outcome = side + 1;
        else if (ply + 1 == kCells) outcome = kDraw;  // discs are never removed: full at ply 42
        ++ply;
        uint64_t t = own; own = opp; opp = t;
        side ^= 1;
    }
    __device__ __forceinline__ void pass() {}
    __device__ __forceinline__ static int canon_of(int b) { return (b >> 3) * 7 + (b & 7); }
    __device__ __forceinline__ static int bit_of(int cell) { return (cell / 7) * 8 + cell % 7; }
    __device__ __forceinline__ static uint64_t canon_word(Mask m, int w) {
        if (w != 0) return 0ull;
        uint64_t out = 0;
#pragma unroll
        for (int r = 0; r < 6; ++r) out |= ((m >> (8 * r)) & 0x7Full) << (7 * r);
        return out;
    }
    static constexpr int kWords = 3;
    __device__ __forceinline__ void save(uint64_t* w) const {
        w[0] = own;
        w[1] = opp;
        w[2] = pack_small(ply, passes, side, outcome);
    }
    __device__ __forceinline__ void load(const uint64_t* w) {
        own = w[0];
        opp = w[1];
        unpack_small(w[2], ply, passes, side, outcome);
    }
};

// --------------------------------------------------------------- Reversi --
template <int S>
__device__ __forceinline__ uint64_t shift64(uint64_t x) {
    return S > 0 ? (x << (S > 0 ? S : 0)) : (x >> (S < 0 ? -S : 0));
}
// Kogge-Stone occluded fill of `gen` through `pro` in direction S (up to 7 steps).
template <int S>
__device__ __forceinline__ uint64_t occluded_fill(uint64_t gen, uint64_t pro) {
    gen |= pro & shift64<S>(gen);
    pro &= shift64<S>(pro);
    gen |= pro & shift64<2 * S>(gen);
    pro &= shift64<2 * S>(pro);
    gen |= pro & shift64<4 * S>(gen);
    return gen;
}

struct Othello {
    static constexpr int kGame = 2, kRows = 8, kCols = 8, kCells = 64, kCap = 128, kPlanes = 2;
    static constexpr bool kHasPass = true;
    static constexpr uint64_t kInner = 0x7E7E7E7E7E7E7E7Eull;  // columns 1..6
    using Mask = uint64_t;
    uint64_t own, opp;
    int side, ply, passes, outcome;

    __device__ __forceinline__ void reset() {
        // D4 (27), E5 (36) white = P2; D5 (35), E4 (28) black = P1; P1 moves.
        own = (1ull << 28) | (1ull << 35);
        opp = (1ull << 27) | (1ull << 36);
        side = ply = passes = 0;
        outcome = kOngoing;
    }
    // cells beyond a run of opponent discs that starts next to one of own's
    template <int S>
    __device__ __forceinline__ static uint64_t dir_moves(uint64_t own, uint64_t pro) {
        return shift64<S>(occluded_fill<S>(own, pro) & pro);
    }
    __device__ __forceinline__ Mask legal() const {
        uint64_t empty = ~(own | opp), ph = opp & kInner;
        uint64_t m = dir_moves<1>(own, ph) | dir_moves<-1>(own, ph) | dir_moves<8>(own, opp) |
                     dir_moves<-8>(own, opp) | dir_moves<7>(own, ph) | dir_moves<-7>(own, ph) |
                     dir_moves<9>(own, ph) | dir_moves<-9>(own, ph);
        return m & empty;
    }
    // opponent discs between x and the first own disc in direction S (or none)
    template <int S>
    __device__ __forceinline__ static uint64_t dir_flips(uint64_t x, uint64_t own, uint64_t pro) {
        uint64_t run = occluded_fill<S>(x, pro) & pro;
        return (shift64<S>(run) & own) ? run : 0ull;
    }
    __device__ __forceinline__ void place(int b) {
        uint64_t x = 1ull << b, ph = opp & kInner;
        uint64_t f = dir_flips<1>(x, own, ph) | dir_flips<-1>(x, own, ph) | dir_flips<8>(x, own, opp) |
                     dir_flips<-8>(x, own, opp) | dir_flips<7>(x, own, ph) | dir_flips<-7>(x, own, ph) |
                     dir_flips<9>(x, own, ph) | dir_flips<-9>(x, own, ph);
        own |= x | f;
        opp &= ~f;
        passes = 0;
        ++ply;
        uint64_t t = own; own = opp; opp = t;
        side ^= 1;
    }
    __device__ __forceinline__ void pass() {
        ++passes;
        ++ply;
        if (passes >= 2) {
            // disc count; own/opp belong to the passing player / the other
            int a = __popcll(own), o = __popcll(opp);
            int winner_is_mover = a > o, winner_is_other = o > a;
            outcome = winner_is_mover ? side + 1 : (winner_is_other ? 2 - side : kDraw);
        }
        uint64_t t = own; own = opp; opp = t;
        side ^= 1;
    }
    __device__ __forceinline__ static int canon_of(int b) { return b; }
    __device__ __forceinline__ static int bit_of(int cell) { return cell; }
    __device__ __forceinline__ static uint64_t canon_word(Mask m, int w) { return w == 0 ? m : 0ull; }
    static constexpr int kWords = 3;
    __device__ __forceinline__ void save(uint64_t* w) const {
        w[0] = own;
        w[1] = opp;
        w[2] = pack_small(ply, passes, side, outcome);
    }
    __device__ __forceinline__ void load(const uint64_t* w) {
        own = w[0];
        opp = w[1];
        unpack_small(w[2], ply, passes, side, outcome);
    }
};

// ------------------------------------------------------------------- Hex --
__host__ __device__ constexpr uint64_t hex_word(int n, int word, int kind) {
    // kind: 0 board, 1 column 0, 2 column n-1, 3 row 0, 4 row n-1
    uint64_t m = 0;
    for (int b = 0; b < 64; ++b) {
        int i = word * 64 + b;
        if (i >= n * n) break;
        int r = i / n, c = i % n;
        bool on = kind == 0 ? true : kind == 1 ? c == 0 : kind == 2 ? c == n - 1 : kind == 3 ? r == 0 : r == n - 1;
        if (on) m |= 1ull << b;
    }
    return m;
}

template <int N>
struct Hex {
    static_assert(N >= 2 && N <= 11, "Hex board 2..11");
    static constexpr int kGame = 3, kRows = N, kCols = N, kCells = N * N, kCap = N * N, kPlanes = 12;
    static constexpr bool kHasPass = false;
    using Mask = B128;
    static constexpr uint64_t kBoardLo = hex_word(N, 0, 0), kBoardHi = hex_word(N, 1, 0);
    static constexpr uint64_t kCol0Lo = hex_word(N, 0, 1), kCol0Hi = hex_word(N, 1, 1);
    static constexpr uint64_t kColLLo = hex_word(N, 0, 2), kColLHi = hex_word(N, 1, 2);
    static constexpr uint64_t kRow0Lo = hex_word(N, 0, 3), kRow0Hi = hex_word(N, 1, 3);
    static constexpr uint64_t kRowLLo = hex_word(N, 0, 4), kRowLHi = hex_word(N, 1, 4);

    B128 own, opp;        // stones
    B128 ownA, ownB;      // own stones connected to own's edge A / edge B
    B128 oppA, oppB;
    B128 front;           // outer layer of the last mover's group still spreading (fused playouts), or empty
    int side, ply, passes, outcome;
    const B128* nbr_table;  // per-cell neighbour masks in shared memory, or nullptr

    __device__ __forceinline__ static B128 board() { return {kBoardLo, kBoardHi}; }
    // a value known to lie on the board: on boards of at most 64 cells the
    // high word is the constant 0, and on 9x9 its upper half is, so the
    // compiler drops every instruction on those words
    __device__ __forceinline__ static B128 fit(B128 a) {
        if constexpr (kBoardHi == 0) return {a.lo, 0ull};
        else if constexpr ((kBoardHi >> 32) == 0) return {a.lo, a.hi & kBoardHi};
        else return a;
    }
    // the six neighbours of the cells of s: (r±1, c), (r, c±1), (r-1, c+1),
    // (r+1, c-1).  A shift by n-1 after a shift by 1 is a shift by n, so the
    // row neighbours ride along with the anti-diagonal ones: four shifts.
    // Shifting by +1 wraps column n-1 onto column 0 of the next row and by -1
    // column 0 onto column n-1, so those results are masked after the shift.
    __device__ __forceinline__ static B128 nbrs(B128 s) {
        const B128 notc0 = {kBoardLo & ~kCol0Lo, kBoardHi & ~kCol0Hi};
        const B128 notcl = {kBoardLo & ~kColLLo, kBoardHi & ~kColLHi};
        const B128 s1 = shl<1>(s), t1 = shr<1>(s);
        const B128 u = s1 | (s & notc0), v = t1 | (s & notcl);
        B128 r = shl<N - 1>(u) | shr<N - 1>(v) | (s1 & notc0) | (t1 & notcl);
        return r & board();
    }
    // edge A / B of the player on `side`: P1 rows 0 and n-1, P2 columns 0 and n-1
    __device__ __forceinline__ static B128 edgeA(int sd) {
        return sd == 0 ? B128{kRow0Lo, kRow0Hi} : B128{kCol0Lo, kCol0Hi};
    }
    __device__ __forceinline__ static B128 edgeB(int sd) {
        return sd == 0 ? B128{kRowLLo, kRowLHi} : B128{kColLLo, kColLHi};
    }
    // stones of `stones` connected to `seed` (seed must be inside stones)
    __device__ __forceinline__ static B128 flood(B128 seed, B128 stones) {
        B128 c = seed;
#pragma unroll 1
        for (int it = 0; it < N * N; ++it) {
            B128 nx = (nbrs(c) & stones) | c;
            if (nx == c) break;
            c = nx;
        }
        return c;
    }
    __device__ __forceinline__ void reset() {
        own = opp = ownA = ownB = oppA = oppB = front = B128{0, 0};
        side = ply = passes = 0;
        outcome = kOngoing;
    }
    __device__ __forceinline__ Mask legal() const { return board() & ~(own | opp); }
    __device__ __forceinline__ void place(int b) {
        B128 x = bit128(b);
        B128 nx = nbr_table ? nbr_table[b] : nbrs(x);
        bool ta = any((x & edgeA(side)) | (nx & ownA));
        bool tb = any((x & edgeB(side)) | (nx & ownB));
        own = own | x;
        if (ta && tb) {
            outcome = side + 1;
        } else if (ta || tb) {
            // the stones newly joined to the touched edge set: x's component
            // among the mover's stones outside both sets, started from x and
            // its neighbours there (nx is at hand), flooded only if there are any
            const B128 stones = own & ~(ownA | ownB), first = nx & stones;
            B128 c = x | first;
            if (any(first)) c = flood(c, stones);
            if (ta) ownA = ownA | c;
            else ownB = ownB | c;
        }
        ++ply;
        B128 t = own; own = opp; opp = t;
        t = ownA; ownA = oppA; oppA = t;
        t = ownB; ownB = oppB; oppB = t;
        side ^= 1;
    }
    __device__ __forceinline__ void pass() {}
    // The same placement with the flood left to spread(): the stone and its
    // neighbours among the mover's stones outside both edge sets join the
    // touched set now, and `front` keeps those neighbours, the layer from
    // which the group goes on growing.  The edge sets are exact again once
    // spread() has returned false; until then no ply may be played.
    __device__ __forceinline__ void place_spread(int b) {
        const B128 x = fit(bit128(b));
        bool ea, eb;
        B128 nx;
        if (nbr_table) {
            const B128 raw = nbr_table[b];
            const uint32_t fl = (uint32_t)(raw.hi >> 60);
            ea = ((side ? fl >> 2 : fl) & 1u) != 0u;
            eb = ((side ? fl >> 3 : fl >> 1) & 1u) != 0u;
            nx = fit(raw);
        } else {
            nx = fit(nbrs(x));
            ea = any(x & edgeA(side));
            eb = any(x & edgeB(side));
        }
        const bool ta = ea || any(nx & ownA);
        const bool tb = eb || any(nx & ownB);
        own = add_disjoint(fit(own), x);
        if (ta && tb) {
            outcome = side + 1;
        } else if (ta || tb) {
            const B128 first = nx & own & ~(ownA | ownB);
            const B128 c = x | first;
            if (ta) ownA = add_disjoint(ownA, c);
            else ownB = add_disjoint(ownB, c);
            front = first;
            passes = ta;  // the set the front joins (kept through the compaction slots with the state)
        }
        ++ply;
        B128 t = own; own = opp; opp = t;
        t = ownA; ownA = oppA; oppA = t;
        t = ownB; ownB = oppB; oppB = t;
        side ^= 1;
    }
    // One layer of the last mover's (now opp's) spreading group: the
    // neighbours of `front` among its stones outside both edge sets join the
    // set that `front` belongs to and become the new front.  The same
    // instructions run whether or not anything is spreading (an empty front
    // adds nothing).  Returns true while the group is still growing.
    __device__ __forceinline__ bool spread() {
        const B128 f = fit(front), a = fit(oppA), b = fit(oppB);
        const bool to_a = passes != 0;  // Hex has no passes: the field says which set the front joins
        const B128 nw = nbrs(f) & fit(opp) & ~add_disjoint(a, b);  // the two edge sets share no stone
        const B128 z = {0ull, 0ull};
        oppA = add_disjoint(a, to_a ? nw : z);
        oppB = add_disjoint(b, to_a ? z : nw);
        front = nw;
        return any(nw);
    }
    // k-th legal cell; on boards of at most 64 cells only the low word
    // exists; otherwise the 32-bit word holding it is found from the words'
    // counts (independent of each other) and the bit inside it by the SWAR
    // search of select_bit
    __device__ __forceinline__ static int pick(B128 m, uint32_t k) {
        if constexpr (kBoardHi == 0) {
            return select_bit(m.lo, k);
        } else {
            const uint32_t w0 = (uint32_t)m.lo, w1 = (uint32_t)(m.lo >> 32), w2 = (uint32_t)m.hi, w3 = (uint32_t)(m.hi >> 32);
            const uint32_t p1 = __popc(w0), p2 = p1 + __popc(w1), p3 = p2 + __popc(w2);
            const bool g1 = k >= p1, g2 = k >= p2, g3 = k >= p3;
            const uint32_t w = g3 ? w3 : (g2 ? w2 : (g1 ? w1 : w0));
            const uint32_t base = g3 ? p3 : (g2 ? p2 : (g1 ? p1 : 0u));
            const int at = (g1 + g2 + g3) * 32;
            return at + select_bit(w, k - base);
        }
    }
    // finish a spreading group (before the state leaves the registers)
    __device__ __forceinline__ void settle() {
#pragma unroll 1
        while (spread()) {
        }
        passes = 0;
    }
    // rebuild the edge-connected sets of both players from the stones
    __device__ __forceinline__ void rebuild() {
        ownA = flood(own & edgeA(side), own);
        ownB = flood(own & edgeB(side), own);
        oppA = flood(opp & edgeA(side ^ 1), opp);
        oppB = flood(opp & edgeB(side ^ 1), opp);
        front = B128{0, 0};
    }
    __device__ __forceinline__ static int canon_of(int b) { return b; }
    __device__ __forceinline__ static int bit_of(int cell) { return cell; }
    __device__ __forceinline__ static uint64_t canon_word(Mask m, int w) { return w == 0 ? m.lo : m.hi; }
    static constexpr int kWords = 15;
    __device__ __forceinline__ void save(uint64_t* w) const {
        w[0] = own.lo; w[1] = own.hi; w[2] = opp.lo; w[3] = opp.hi;
        w[4] = ownA.lo; w[5] = ownA.hi; w[6] = ownB.lo; w[7] = ownB.hi;
        w[8] = oppA.lo; w[9] = oppA.hi; w[10] = oppB.lo; w[11] = oppB.hi;
        w[12] = pack_small(ply, passes, side, outcome);
        w[13] = front.lo; w[14] = front.hi;
    }
    __device__ __forceinline__ void load(const uint64_t* w) {
        own = {w[0], w[1]}; opp = {w[2], w[3]};
        ownA = {w[4], w[5]}; ownB = {w[6], w[7]};
        oppA = {w[8], w[9]}; oppB = {w[10], w[11]};
        unpack_small(w[12], ply, passes, side, outcome);
        front = {w[13], w[14]};
    }
};

// Fill a shared-memory table of per-cell neighbour masks for Hex<N>
// (cooperatively by the block; caller synchronises).  The four top bits of
// an entry (bits 124..127, never cells: n*n <= 121) say whether the cell is
// on row 0, row n-1, column 0, column n-1 -- the players' edges -- so a
// placement reads its edge contacts with its neighbours.
template <int N>
__device__ __forceinline__ void hex_fill_table(B128* table) {
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
        B128 m = Hex<N>::nbrs(bit128(i));
        const int r = i / N, c = i % N;
        m.hi |= ((uint64_t)(r == 0) << 60) | ((uint64_t)(r == N - 1) << 61) | ((uint64_t)(c == 0) << 62) |
                ((uint64_t)(c == N - 1) << 63);
        table[i] = m;
    }
}

// ------------------------------------------------- multi-word bitboards --
template <int W>
struct BitsW {
    uint64_t w[W];
};
template <int W>
__device__ __forceinline__ BitsW<W> operator|(const BitsW<W>& a, const BitsW<W>& b) {
    BitsW<W> o;
#pragma unroll
    for (int i = 0; i < W; ++i) o.w[i] = a.w[i] | b.w[i];
    return o;
}
template <int W>
__device__ __forceinline__ BitsW<W> operator&(const BitsW<W>& a, const BitsW<W>& b) {
    BitsW<W> o;
#pragma unroll
    for (int i = 0; i < W; ++i) o.w[i] = a.w[i] & b.w[i];
    return o;
}
template <int W>
__device__ __forceinline__ BitsW<W> operator~(const BitsW<W>& a) {
    BitsW<W> o;
#pragma unroll
    for (int i = 0; i < W; ++i) o.w[i] = ~a.w[i];
    return o;
}
template <int W>
__device__ __forceinline__ bool any(const BitsW<W>& a) {
    uint64_t x = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) x |= a.w[i];
    return x != 0;
}
template <int W>
__device__ __forceinline__ uint32_t popc(const BitsW<W>& a) {
    uint32_t n = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) n += __popcll(a.w[i]);
    return n;
}
// bit i of the result = bit i + S of a (S >= 0, compile time)
template <int S, int W>
__device__ __forceinline__ BitsW<W> shr(const BitsW<W>& a) {
    constexpr int q = S / 64, r = S % 64;
    BitsW<W> o;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const uint64_t lo = (i + q < W) ? a.w[i + q] : 0ull;
        const uint64_t hi = (i + q + 1 < W) ? a.w[i + q + 1] : 0ull;
        o.w[i] = r == 0 ? lo : ((lo >> (r == 0 ? 1 : r)) | (hi << (r == 0 ? 1 : 64 - r)));
    }
    return o;
}
// bit i of the result = bit i - S of a
template <int S, int W>
__device__ __forceinline__ BitsW<W> shl(const BitsW<W>& a) {
    constexpr int q = S / 64, r = S % 64;
    BitsW<W> o;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const uint64_t hi = (i - q >= 0) ? a.w[i - q] : 0ull;
        const uint64_t lo = (i - q - 1 >= 0) ? a.w[i - q - 1] : 0ull;
        o.w[i] = r == 0 ? hi : ((hi << (r == 0 ? 1 : r)) | (lo >> (r == 0 ? 1 : 64 - r)));
    }
    return o;
}
// dynamic single-bit access without indexing the register array (p may lie
// outside the board: the test then reads 0)
template <int W>
__device__ __forceinline__ bool test_bit(const BitsW<W>& a, int p) {
    uint64_t word = 0;
    const int q = p >> 6;
#pragma unroll
    for (int i = 0; i < W; ++i) word = q == i ? a.w[i] : word;
    return p >= 0 && ((word >> (p & 63)) & 1ull);
}
template <int W>
__device__ __forceinline__ void set_bit_w(BitsW<W>& a, int p) {
    const int q = p >> 6;
    const uint64_t b = 1ull << (p & 63);
#pragma unroll
    for (int i = 0; i < W; ++i) a.w[i] |= q == i ? b : 0ull;
}
template <int W>
__device__ __forceinline__ void clear_bit_w(BitsW<W>& a, int p) {
    const int q = p >> 6;
    const uint64_t b = 1ull << (p & 63);
#pragma unroll
    for (int i = 0; i < W; ++i) a.w[i] &= q == i ? ~b : ~0ull;
}
template <int W>
__device__ __forceinline__ int select_bit(const BitsW<W>& m, uint32_t k) {
    uint32_t pre = 0, base = 0;
    uint64_t word = m.w[0];
    int widx = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const uint32_t c = __popcll(m.w[i]);
        const bool here = k >= pre && k < pre + c;
        word = here ? m.w[i] : word;
        base = here ? pre : base;
        widx = here ? i : widx;
        pre += c;
    }
    return widx * 64 + select_bit(word, k - base);
}
template <int W>
__device__ __forceinline__ BitsW<W> bits_from(const uint64_t (&v)[W]) {
    BitsW<W> o;
#pragma unroll
    for (int i = 0; i < W; ++i) o.w[i] = v[i];
    return o;
}

// word `word` of the mask of cells (r < R, c < C) in a row-stride-S layout,
// optionally restricted to the hexagon |r - c| <= 4
__host__ __device__ constexpr uint64_t grid_word(int R, int C, int S, bool hexagon, int word) {
    uint64_t m = 0;
    for (int b = 0; b < 64; ++b) {
        int i = word * 64 + b, r = i / S, c = i % S;
        if (r < R && c < C && (!hexagon || (r - c <= 4 && c - r <= 4))) m |= 1ull << b;
    }
    return m;
}

// any run of >= 5 (L5) / >= 4 / >= 3 stones along stride D, full board
template <int D, int W>
__device__ __forceinline__ BitsW<W> runs2(const BitsW<W>& b) { return b & shr<D>(b); }
template <int D, int W>
__device__ __forceinline__ bool has_run5(const BitsW<W>& b) {
    const BitsW<W> m2 = runs2<D>(b), m4 = m2 & shr<2 * D>(m2);
    return any(m4 & shr<4 * D>(b));
}
// a maximal run of exactly five: starts of >= 5 windows with no stone before
// the window and none right after it
template <int D, int W>
__device__ __forceinline__ bool has_exact5(const BitsW<W>& b) {
    const BitsW<W> m2 = runs2<D>(b), m4 = m2 & shr<2 * D>(m2), m5 = m4 & shr<4 * D>(b);
    return any(m5 & ~shl<D>(b) & ~shr<5 * D>(b));
}

// ------------------------------------------------------------- Gomoku --
struct Gomoku {
    static constexpr int kGame = 4, kRows = 15, kCols = 15, kCells = 225, kCap = 225, W = 4, kStride = 16;
    static constexpr int kPlanes = 2 * W;
    static constexpr bool kHasPass = false;
    using Mask = BitsW<W>;
    Mask own, opp;
    int side, ply, passes, outcome;

    __device__ __forceinline__ static Mask valid() {
        return Mask{{grid_word(15, 15, 16, false, 0), grid_word(15, 15, 16, false, 1), grid_word(15, 15, 16, false, 2),
                     grid_word(15, 15, 16, false, 3)}};
    }
    __device__ __forceinline__ void reset() {
        own = opp = Mask{{0, 0, 0, 0}};
        side = ply = passes = 0;
        outcome = kOngoing;
    }
    __device__ __forceinline__ Mask legal() const { return valid() & ~(own | opp); }
    __device__ __forceinline__ static bool five(const Mask& b) {
        return has_exact5<1>(b) | has_exact5<16>(b) | has_exact5<17>(b) | has_exact5<15>(b);
    }
    __device__ __forceinline__ void place(int b) {
        set_bit_w(own, b);
        if (five(own)) outcome = side + 1;
        else if (ply + 1 >= kCells) outcome = kDraw;
        ++ply;
        Mask t = own; own = opp; opp = t;
        side ^= 1;
    }
    __device__ __forceinline__ void pass() {}
    __device__ __forceinline__ static int canon_of(int b) { return (b >> 4) * 15 + (b & 15); }
    __device__ __forceinline__ static int bit_of(int cell) { return (cell / 15) * 16 + cell % 15; }
    static constexpr int kWords = 2 * W + 1;
    __device__ __forceinline__ void save(uint64_t* w) const {
#pragma unroll
        for (int i = 0; i < W; ++i) { w[i] = own.w[i]; w[W + i] = opp.w[i]; }
        w[2 * W] = pack_small(ply, passes, side, outcome);
    }
    __device__ __forceinline__ void load(const uint64_t* w) {
#pragma unroll
        for (int i = 0; i < W; ++i) { own.w[i] = w[i]; opp.w[i] = w[W + i]; }
        unpack_small(w[2 * W], ply, passes, side, outcome);
    }
};

// --------------------------------------------------------------- Pente --
struct Pente {
    static constexpr int kGame = 5, kRows = 19, kCols = 19, kCells = 361, kCap = 2000, W = 6, kStride = 20;
    static constexpr int kPlanes = 2 * W;
    static constexpr bool kHasPass = false;
    static constexpr int kCentre = 9 * 20 + 9;
    using Mask = BitsW<W>;
    Mask own, opp;
    int side, ply, passes, outcome;
    int caps_own, caps_opp;  // pairs captured by the player to move / by the other

    __device__ __forceinline__ static Mask valid() {
        return Mask{{grid_word(19, 19, 20, false, 0), grid_word(19, 19, 20, false, 1), grid_word(19, 19, 20, false, 2),
                     grid_word(19, 19, 20, false, 3), grid_word(19, 19, 20, false, 4), grid_word(19, 19, 20, false, 5)}};
    }
    __device__ __forceinline__ void reset() {
        own = opp = Mask{{0, 0, 0, 0, 0, 0}};
        side = ply = passes = 0;
        caps_own = caps_opp = 0;
        outcome = kOngoing;
    }
    __device__ __forceinline__ Mask legal() const {
        if (ply == 0) {
            Mask c = Mask{{0, 0, 0, 0, 0, 0}};
            set_bit_w(c, kCentre);
            return c & ~(own | opp);
        }
        return valid() & ~(own | opp);
    }
    // own - opp - opp - own along D from the new stone b: remove the pair
    template <int D>
    __device__ __forceinline__ void capture(int b) {
        if (test_bit(opp, b + D) && test_bit(opp, b + 2 * D) && test_bit(own, b + 3 * D)) {
            clear_bit_w(opp, b + D);
            clear_bit_w(opp, b + 2 * D);
            ++caps_own;
        }
    }
    __device__ __forceinline__ static bool five(const Mask& b) {
        return has_run5<1>(b) | has_run5<20>(b) | has_run5<21>(b) | has_run5<19>(b);
    }
    __device__ __forceinline__ void place(int b) {
        set_bit_w(own, b);
        capture<1>(b);
        capture<-1>(b);
        capture<20>(b);
        capture<-20>(b);
        capture<21>(b);
        capture<-21>(b);
        capture<19>(b);
        capture<-19>(b);
        if (five(own) || caps_own >= 5) outcome = side + 1;
        else if (!any(valid() & ~(own | opp))) outcome = kDraw;
        ++ply;
        Mask t = own; own = opp; opp = t;
        int c = caps_own; caps_own = caps_opp; caps_opp = c;
        side ^= 1;
    }
    __device__ __forceinline__ void pass() {}
    __device__ __forceinline__ static int canon_of(int b) { return (b / 20) * 19 + b % 20; }
    __device__ __forceinline__ static int bit_of(int cell) { return (cell / 19) * 20 + cell % 19; }
    static constexpr int kWords = 2 * W + 1;
    __device__ __forceinline__ void save(uint64_t* w) const {
#pragma unroll
        for (int i = 0; i < W; ++i) { w[i] = own.w[i]; w[W + i] = opp.w[i]; }
        w[2 * W] = pack_small(ply, passes, side, outcome) | ((uint64_t)(caps_own & 15) << 40) |
                   ((uint64_t)(caps_opp & 15) << 44);
    }
    __device__ __forceinline__ void load(const uint64_t* w) {
#pragma unroll
        for (int i = 0; i < W; ++i) { own.w[i] = w[i]; opp.w[i] = w[W + i]; }
        unpack_small(w[2 * W] & 0xFFFFFFFFFFull, ply, passes, side, outcome);
        caps_own = (int)((w[2 * W] >> 40) & 15);
        caps_opp = (int)((w[2 * W] >> 44) & 15);
    }
};

// ------------------------------------------------------------ Yavalath --
struct Yavalath {
    static constexpr int kGame = 6, kRows = 9, kCols = 9, kCells = 61, kCap = 61, W = 2, kStride = 10;
    static constexpr int kPlanes = 2 * W;
    static constexpr bool kHasPass = false;
    using Mask = BitsW<W>;
    Mask own, opp;
    int side, ply, passes, outcome;

    __device__ __forceinline__ static Mask valid() {
        return Mask{{grid_word(9, 9, 10, true, 0), grid_word(9, 9, 10, true, 1)}};
    }
    __device__ __forceinline__ void reset() {
        own = opp = Mask{{0, 0}};
        side = ply = passes = 0;
        outcome = kOngoing;
    }
    __device__ __forceinline__ Mask legal() const { return valid() & ~(own | opp); }
    template <int D>
    __device__ __forceinline__ static bool run4(const Mask& b) {
        const Mask m2 = runs2<D>(b);
        return any(m2 & shr<2 * D>(m2));
    }
    template <int D>
    __device__ __forceinline__ static bool run3(const Mask& b) {
        return any(runs2<D>(b) & shr<2 * D>(b));
    }
    __device__ __forceinline__ void place(int b) {
        set_bit_w(own, b);
        // the hexagon's three axes: strides 1, 10 and 11 in the axial layout
        if (run4<1>(own) | run4<10>(own) | run4<11>(own)) outcome = side + 1;
        else if (run3<1>(own) | run3<10>(own) | run3<11>(own)) outcome = 2 - side;  // three without four loses
        else if (ply + 1 >= kCells) outcome = kDraw;
        ++ply;
        Mask t = own; own = opp; opp = t;
        side ^= 1;
    }
    __device__ __forceinline__ void pass() {}
    // canonical id <-> axial (r, c): rows of 5,6,7,8,9,8,7,6,5 cells; c starts at max(0, r-4)
    __device__ __forceinline__ static int bit_of(int cell) {
        int r = 0, start = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int len = 9 - (i > 4 ? i - 4 : 4 - i);
            const bool past = cell >= start + len && r == i;
            start += past ? len : 0;
            r += past ? 1 : 0;
        }
        return r * 10 + (cell - start) + (r > 4 ? r - 4 : 0);
    }
    __device__ __forceinline__ static int canon_of(int b) {
        const int r = b / 10, c = b % 10;
        int start = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) start += i < r ? 9 - (i > 4 ? i - 4 : 4 - i) : 0;
        return start + c - (r > 4 ? r - 4 : 0);
    }
    static constexpr int kWords = 2 * W + 1;
    __device__ __forceinline__ void save(uint64_t* w) const {
        w[0] = own.w[0]; w[1] = own.w[1]; w[2] = opp.w[0]; w[3] = opp.w[1];
        w[4] = pack_small(ply, passes, side, outcome);
    }
    __device__ __forceinline__ void load(const uint64_t* w) {
        own = Mask{{w[0], w[1]}};
        opp = Mask{{w[2], w[3]}};
        unpack_small(w[4], ply, passes, side, outcome);
    }
};

// ------------------------------------------------ parametric line game --
// Any R x C board with R * (C + 1) <= 128 in a stride C + 1 layout (two
// words): place on an empty cell -- with Connect-Four gravity if asked -- and
// a line of at least L (or exactly L) stones along a row, column or diagonal
// wins, or loses in the misere variant; a full board draws.  All parameters
// come from the env's descriptor at run time.
// 64-bit shifts with PTX semantics: an amount of 64 or more (as unsigned)
// gives 0, so the 128-bit shifts below need no branch on the amount
__device__ __forceinline__ uint64_t shr64c(uint64_t x, uint32_t s) {
    uint64_t r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
    return r;
}
__device__ __forceinline__ uint64_t shl64c(uint64_t x, uint32_t s) {
    uint64_t r;
    asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
    return r;
}
// bit i of the result = bit i + s of a (0 <= s, run-time; 64 - s and s - 64
// wrap to large unsigned amounts, which give 0)
__device__ __forceinline__ BitsW<2> shr_rt(const BitsW<2>& a, int s) {
    const uint32_t u = (uint32_t)s;
    BitsW<2> o;
    o.w[0] = shr64c(a.w[0], u) | shl64c(a.w[1], 64u - u) | shr64c(a.w[1], u - 64u);
    o.w[1] = shr64c(a.w[1], u);
    return o;
}
// bit i of the result = bit i - s of a
__device__ __forceinline__ BitsW<2> shl_rt(const BitsW<2>& a, int s) {
    const uint32_t u = (uint32_t)s;
    BitsW<2> o;
    o.w[1] = shl64c(a.w[1], u) | shr64c(a.w[0], 64u - u) | shl64c(a.w[0], u - 64u);
    o.w[0] = shl64c(a.w[0], u);
    return o;
}

struct LineGame {
    static constexpr int kGame = 7, kRows = 0, kCols = 0, kCells = 128, kCap = 128, W = 2, kPlanes = 4;
    static constexpr bool kHasPass = false;
    static constexpr int kExact = 1, kGravity = 2, kMisere = 4;
    using Mask = BitsW<2>;
    Mask own, opp;
    int side, ply, passes, outcome;
    int R, C, S, L, flags;
    Mask valid, bottom;

    // parameters from a descriptor: game | R << 8 | C << 16 | L << 24 | flags << 28
    __device__ __forceinline__ void configure(int32_t desc) {
        R = (desc >> 8) & 0xFF;
        C = (desc >> 16) & 0xFF;
        L = (desc >> 24) & 15;
        flags = (desc >> 28) & 7;
        S = C + 1;
        const uint64_t row = (C >= 64) ? ~0ull : ((1ull << C) - 1ull);
        valid = Mask{{0, 0}};
        for (int r = 0; r < R; ++r) valid = valid | shl_rt(Mask{{row, 0}}, r * S);
        bottom = shl_rt(Mask{{row, 0}}, (R - 1) * S);
    }
    __device__ __forceinline__ int cells() const { return R * C; }
    __device__ __forceinline__ void reset() {
        own = opp = Mask{{0, 0}};
        side = ply = passes = 0;
        outcome = kOngoing;
    }
    __device__ __forceinline__ Mask legal() const {
        const Mask occ = own | opp;
        Mask m = valid & ~occ;
        if (flags & kGravity) m = m & (shr_rt(occ, S) | bottom);
        return m;
    }
    // a run of L stones along step d, by doubling: after the loop bit i of m
    // is set iff cells i, i+d, ..., i+(k-1)d all hold a stone (k < L < 2k),
    // and the last shift by (L-k)d closes the window to L cells
    __device__ __forceinline__ bool line_dir(const Mask& b, int d) const {
        Mask m = b;
        int k = 1;
        for (; 2 * k <= L; k *= 2) m = m & shr_rt(m, k * d);
        if (k < L) m = m & shr_rt(m, (L - k) * d);
        if (flags & kExact) m = m & ~shl_rt(b, d) & ~shr_rt(b, L * d);
        return any(m);
    }
    __device__ __forceinline__ void place(int b) {
        set_bit_w(own, b);
        const bool made = line_dir(own, 1) | line_dir(own, S) | line_dir(own, S + 1) | line_dir(own, S - 1);
        // no stone is ever removed, so the board is full at ply R*C
        if (made) outcome = (flags & kMisere) ? 2 - side : side + 1;
        else if (ply + 1 == R * C) outcome = kDraw;
        ++ply;
        Mask t = own; own = opp; opp = t;
        side ^= 1;
    }
    __device__ __forceinline__ void pass() {}
    __device__ __forceinline__ int canon_of(int b) const { return (b / S) * C + b % S; }
    __device__ __forceinline__ int bit_of(int cell) const { return (cell / C) * S + cell % C; }
    static constexpr int kWords = 5;
    __device__ __forceinline__ void save(uint64_t* w) const {
        w[0] = own.w[0]; w[1] = own.w[1]; w[2] = opp.w[0]; w[3] = opp.w[1];
        w[4] = pack_small(ply, passes, side, outcome);
    }
    __device__ __forceinline__ void load(const uint64_t* w) {
        own = Mask{{w[0], w[1]}};
        opp = Mask{{w[2], w[3]}};
        unpack_small(w[4], ply, passes, side, outcome);
    }
};

}  // namespace ludax
#include "ludax_movegames.cuh"
namespace ludax {

// parameters of a game instance: no-ops except for the parametric line game
template <class G>
__device__ __forceinline__ void configure(G& g, int32_t desc) {
    if constexpr (G::kGame == LineGame::kGame) g.configure(desc);
}
template <class G>
__device__ __forceinline__ int cells_of(const G& g) {
    if constexpr (G::kGame == LineGame::kGame) return g.cells();
    else return G::kCells;
}

// Games that keep derived data with their state (C4's next legal cells,
// Draughts' legal count) rebuild it with refresh() after a position is
// loaded; the others have nothing to rebuild.
template <class G, class = void>
struct HasRefresh : std::false_type {};
template <class G>
struct HasRefresh<G, std::void_t<decltype(std::declval<G&>().refresh())>> : std::true_type {};
template <class G>
__device__ __forceinline__ void refresh_of(G& g) {
    if constexpr (HasRefresh<G>::value) g.refresh();
}
// number of legal actions in the mask m = g.legal()
template <class G, class = void>
struct HasLegalCount : std::false_type {};
template <class G>
struct HasLegalCount<G, std::void_t<decltype(std::declval<const G&>().legal_count())>> : std::true_type {};
template <class G>
__device__ __forceinline__ uint32_t legal_count_of(const G& g, const typename G::Mask& m) {
    if constexpr (HasLegalCount<G>::value) return g.legal_count();
    else return popc(m);
}

// Games whose legal mask is ordinal (kOrdinal: bits 0 .. count() - 1, one
// per legal action in action order): the k-th legal action is k itself, so
// a random ply needs only the count, not the mask.
template <class G, class = void>
struct IsOrdinal : std::false_type {};
template <class G>
struct IsOrdinal<G, std::enable_if_t<G::kOrdinal>> : std::true_type {};

// Games whose placement can leave a flood to spread over later loop steps
// (Hex in the fused playouts): place_spread(), spread(), settle().
template <class G, class = void>
struct HasSpread : std::false_type {};
template <class G>
struct HasSpread<G, std::void_t<decltype(std::declval<G&>().spread())>> : std::true_type {};
// bring a state whose flood may still be spreading to its exact form
template <class G>
__device__ __forceinline__ void settle_of(G& g) {
    if constexpr (HasSpread<G>::value) g.settle();
}

// ---------------------------------------------------------- one random ply --
// Uniform-random policy: n legal cells, k-th in ascending cell id with
// k = umulhi(top32(sm(key ^ ply)), n); a forced pass draws nothing.
template <class G>
__device__ __forceinline__ void random_ply(G& g, uint64_t key) {
    if constexpr (IsOrdinal<G>::value) {  // no pass in these games; called only while the game is on
        g.place((int)draw_index(key, (uint32_t)g.ply, (uint32_t)g.count()));
        if (g.outcome == kOngoing && g.ply >= G::kCap) g.outcome = kCapped;
        return;
    }
    typename G::Mask m = g.legal();
    if (G::kHasPass && !any(m)) {
        g.pass();
    } else {
        uint32_t k = draw_index(key, (uint32_t)g.ply, legal_count_of(g, m));
        g.place(select_bit(m, k));
    }
    if (g.outcome == kOngoing && g.ply >= G::kCap) g.outcome = kCapped;
}

// The same ply taken by all 32 lanes of a warp that hold the same position
// (the UCT kernel, where a warp owns one search): games with a warp form of
// the move lookup (place_warp) share its work across the lanes; the others
// compute it in every lane.  Every lane ends with the same state.
template <class G, class = void>
struct HasWarpPlace : std::false_type {};
template <class G>
struct HasWarpPlace<G, std::void_t<decltype(std::declval<G&>().place_warp(0, 0))>> : std::true_type {};
template <class G>
__device__ __forceinline__ void random_ply_warp(G& g, uint64_t key, int lane) {
    if constexpr (HasWarpPlace<G>::value && IsOrdinal<G>::value) {
        g.place_warp((int)draw_index(key, (uint32_t)g.ply, (uint32_t)g.count()), lane);
        if (g.outcome == kOngoing && g.ply >= G::kCap) g.outcome = kCapped;
    } else if constexpr (HasWarpPlace<G>::value) {
        typename G::Mask m = g.legal();
        if (G::kHasPass && !any(m)) {
            g.pass();
        } else {
            g.place_warp((int)draw_index(key, (uint32_t)g.ply, legal_count_of(g, m)), lane);
        }
        if (g.outcome == kOngoing && g.ply >= G::kCap) g.outcome = kCapped;
    } else {
        random_ply(g, key);
    }
}

// The same ply with the draw software-pipelined: rhi holds the top 32 bits of
// this ply's draw (computed one ply ahead); the next ply's draw is started
// here, independent of the board work, and handed back through rhi.  The
// result is identical to random_ply.
__device__ __forceinline__ uint32_t draw_hi(uint64_t key, uint32_t ply) {
    return (uint32_t)(splitmix64(key ^ (uint64_t)ply) >> 32);
}
// Games with a spreading flood (HasSpread) first grow it by one layer; while
// it still grows the env plays no ply this step (its edge sets are not yet
// exact), so every ply sees the same state as with the eager flood.
template <class G>
__device__ __forceinline__ void random_ply_pre(G& g, uint64_t key, uint32_t& rhi) {
    if constexpr (HasSpread<G>::value) {
        if (g.spread()) return;
        const uint32_t rnext = draw_hi(key, (uint32_t)g.ply + 1u);
        const typename G::Mask m = g.legal();
        g.place_spread(G::pick(m, __umulhi(rhi, popc(m))));
        if (g.outcome == kOngoing && g.ply >= G::kCap) g.outcome = kCapped;
        rhi = rnext;
        return;
    }
    const uint32_t rnext = draw_hi(key, (uint32_t)g.ply + 1u);
    if constexpr (IsOrdinal<G>::value) {
        g.place((int)__umulhi(rhi, (uint32_t)g.count()));
    } else {
        typename G::Mask m = g.legal();
        if (G::kHasPass && !any(m)) {
            g.pass();
        } else {
            g.place(select_bit(m, __umulhi(rhi, legal_count_of(g, m))));
        }
    }
    if (g.outcome == kOngoing && g.ply >= G::kCap) g.outcome = kCapped;
    rhi = rnext;
}

}  // namespace ludax
