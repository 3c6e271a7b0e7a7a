// ludax_movegames.cuh -- games whose pieces move (App. C): Wolf and Sheep,
// English Draughts, Dai Hasami Shogi.
//
// An action is from * cells + to (canonical cells, row 0 at the top).  The
// kernels see a move game through the same interface as a placement game:
// legal() returns an "ordinal mask" whose n lowest bits are set, n = the
// number of legal actions, and place(k) plays the k-th legal action in
// ascending action id.  So the uniform-random ply (k-th of n by the draw)
// and the tree search (tried sets over ordinals) run unchanged.  The k-th
// action is found by walking the mover's pieces in ascending cell order with
// each piece's destination bitboard (ascending destination = ascending
// action id, because every internal layout is monotone in the cell id).
//
// Pieces are kept per player (P1 = index 0, starting at the bottom and moving
// up); the state view's cell values are 1 / 2 for a piece of P1 / P2 and
// 3 / 4 for a Draughts king of P1 / P2.  In all three games the mover wins
// when the player to move next has no legal action; the ply cap is 200
// (Sec. 6 stops games of unbounded length after 200 turns).
#pragma once

namespace ludax {

template <class G>
struct IsMove {
    static constexpr bool value = false;
};

__device__ __forceinline__ uint32_t ordinals32(int n) { return n >= 32 ? 0xFFFFFFFFu : ((1u << n) - 1u); }
__device__ __forceinline__ uint64_t ordinals64(int n) { return n >= 64 ? ~0ull : (n <= 0 ? 0ull : ((1ull << n) - 1ull)); }
template <int W>
__device__ __forceinline__ BitsW<W> ordinalsW(int n) {
    BitsW<W> m;
#pragma unroll
    for (int i = 0; i < W; ++i) m.w[i] = ordinals64(n - 64 * i);
    return m;
}
__device__ __forceinline__ int lowest(uint64_t m) { return __ffsll((long long)m) - 1; }

// diagonal steps on an 8x8 board, cell = r * 8 + c: 0 up-left, 1 up-right,
// 2 down-left, 3 down-right (the file masks stop wrap-around)
constexpr uint64_t kNotFileA = 0xFEFEFEFEFEFEFEFEull, kNotFileH = 0x7F7F7F7F7F7F7F7Full;
__device__ __forceinline__ uint64_t diag_step(uint64_t b, int d) {
    switch (d) {
    case 0: return (b & kNotFileA) >> 9;
    case 1: return (b & kNotFileH) >> 7;
    case 2: return (b & kNotFileA) << 7;
    default: return (b & kNotFileH) << 9;
    }
}

// ------------------------------------------------------ Wolf and Sheep --
// Four sheep (P1) start on the dark cells of the bottom row and step
// diagonally forward; the wolf (P2) starts on cell 3 (the left one of the
// two central dark cells of the top row) and steps diagonally either way;
// the wolf wins on the bottom row.
struct WolfSheep {
    static constexpr int kGame = 8, kRows = 8, kCols = 8, kCells = 64, kCap = 200, kPlanes = 2, kActions = 4096;
    static constexpr bool kHasPass = false;
    static constexpr bool kOrdinal = true;  // legal() holds the ordinals 0 .. count() - 1
    using Mask = uint32_t;  // ordinals: at most 8 legal actions
    uint64_t own, opp;      // pieces of the side to move / of the other side
    int side, ply, passes, outcome;

    __device__ __forceinline__ void reset() {
        own = (1ull << 56) | (1ull << 58) | (1ull << 60) | (1ull << 62);
        opp = 1ull << 3;
        side = ply = passes = 0;
        outcome = kOngoing;
    }
    // destinations of the mover's piece on cell i (sheep: up only)
    __device__ __forceinline__ uint64_t dests(int i) const {
        const uint64_t b = 1ull << i, empty = ~(own | opp);
        uint64_t d = diag_step(b, 0) | diag_step(b, 1);
        if (side == 1) d |= diag_step(b, 2) | diag_step(b, 3);
        return d & empty;
    }
    __device__ __forceinline__ int count() const {
        int n = 0;
        for (uint64_t m = own; m; m &= m - 1) n += __popcll(dests(lowest(m)));
        return n;
    }
    __device__ __forceinline__ Mask legal() const { return ordinals32(count()); }
    __device__ __forceinline__ void find(int k, int& from, int& to) const {
        from = to = -1;
        for (uint64_t m = own; m; m &= m - 1) {
            const int i = lowest(m);
            const uint64_t d = dests(i);
            const int c = __popcll(d);
            if (k < c) {
                from = i;
                to = select_bit(d, (uint32_t)k);
                return;
            }
            k -= c;
        }
    }
    __device__ __forceinline__ void place(int k) {
        int f, t;
        find(k, f, t);
        const int p = side;
        own ^= (1ull << f) | (1ull << t);
        const uint64_t x = own;
        own = opp;
        opp = x;
        ++ply;
        side ^= 1;
        if (p == 1 && t >= 56) outcome = kWin2;
        else if (count() == 0) outcome = p + 1;
    }
    __device__ __forceinline__ void pass() {}
    __device__ __forceinline__ int canon_of(int k) const {
        int f, t;
        find(k, f, t);
        return f * kCells + t;
    }
    // ordinal of the canonical action a, -1 if it is not legal
    __device__ __forceinline__ int bit_of(int a) const {
        const int f = a / kCells, t = a % kCells;
        if (!((own >> f) & 1)) return -1;
        int base = 0;
        for (uint64_t m = own & ((1ull << f) - 1); m; m &= m - 1) base += __popcll(dests(lowest(m)));
        const uint64_t d = dests(f);
        if (!((d >> t) & 1)) return -1;
        return base + __popcll(d & ((1ull << t) - 1));
    }
    template <class F>
    __device__ __forceinline__ void for_each_move(F&& f) const {
        for (uint64_t m = own; m; m &= m - 1) {
            const int i = lowest(m);
            for (uint64_t d = dests(i); d; d &= d - 1) f(i * kCells + lowest(d));
        }
    }
    __device__ __forceinline__ uint64_t occupied() const { return own | opp; }
    __device__ __forceinline__ uint64_t p1() const { return side == 0 ? own : opp; }
    __device__ __forceinline__ uint64_t p2() const { return side == 0 ? opp : own; }
    __device__ __forceinline__ void clear() { own = opp = 0; }
    __device__ __forceinline__ int cell_value(int i) const {
        return ((p1() >> i) & 1) ? 1 : (((p2() >> i) & 1) ? 2 : 0);
    }
    // absolute placement: call with side already set
    __device__ __forceinline__ void set_cell(int i, int v) {
        if (v == 1) (side == 0 ? own : opp) |= 1ull << i;
        if (v == 2) (side == 0 ? opp : own) |= 1ull << i;
    }
    __device__ __forceinline__ int extra() const { return 0; }
    __device__ __forceinline__ void set_extra(int) {}
    __device__ __forceinline__ void refresh() {}
    __device__ __forceinline__ void planes_out(uint64_t* w) const {
        w[0] = p1();
        w[1] = p2();
    }
    __device__ __forceinline__ void planes_in(const uint64_t* w) {  // side already set
        own = side == 0 ? w[0] : w[1];
        opp = side == 0 ? w[1] : w[0];
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
template <>
struct IsMove<WolfSheep> {
    static constexpr bool value = true;
};

// --------------------------------------------------- English Draughts --
// Men on the dark cells ((r + c) odd), P1 on rows 5-7, P2 on rows 0-2.  Men
// step diagonally forward, kings either way; a hop over an adjacent opposing
// piece onto the empty cell beyond removes it; while any hop exists only
// hops are legal; a man ending on the far row is crowned; after a hop the
// same player moves again, with that piece's hops only, while it has one.
struct Draughts {
    static constexpr int kGame = 9, kRows = 8, kCols = 8, kCells = 64, kCap = 200, kPlanes = 4, kActions = 4096;
    static constexpr bool kHasPass = false;
    static constexpr bool kOrdinal = true;  // legal() holds the ordinals 0 .. count() - 1
    using Mask = uint64_t;  // ordinals: at most 48 legal actions (12 pieces x 4 directions)
    uint64_t men_own, kings_own, men_opp, kings_opp;  // relative to the side to move
    int side, ply, passes, outcome, pending;           // pending: cell of the piece that must hop again, -1 if none
    int ncache;                                        // legal actions of the position (refresh())
    bool capcache;                                     // whether they are hops
    uint64_t src[4];                                   // per direction, the movers that have that move (refresh())

    __device__ __forceinline__ void reset() {
        men_own = 0x55AA550000000000ull;  // P1: dark cells of rows 5-7
        men_opp = 0x0000000000AA55AAull;  // P2: dark cells of rows 0-2
        kings_own = kings_opp = 0;
        side = ply = passes = 0;
        pending = -1;
        outcome = kOngoing;
        refresh();
    }
    __device__ __forceinline__ uint64_t own() const { return men_own | kings_own; }
    __device__ __forceinline__ uint64_t opp() const { return men_opp | kings_opp; }
    __device__ __forceinline__ uint64_t empty() const { return ~(own() | opp()); }
    // may the mover's piece on cell i move in direction d?  (men of P1 go
    // up: 0, 1; men of P2 down: 2, 3; kings both)
    __device__ __forceinline__ bool moves_in(int i, int d) const {
        return ((kings_own >> i) & 1) || (side == 0 ? d < 2 : d >= 2);
    }
    __device__ __forceinline__ uint64_t hops_of(int i) const {
        const uint64_t b = 1ull << i, e = empty(), o = opp();
        uint64_t r = 0;
#pragma unroll
        for (int d = 0; d < 4; ++d)
            if (moves_in(i, d)) r |= diag_step(diag_step(b, d) & o, d) & e;
        return r;
    }
    __device__ __forceinline__ uint64_t steps_of(int i) const {
        const uint64_t b = 1ull << i, e = empty();
        uint64_t r = 0;
#pragma unroll
        for (int d = 0; d < 4; ++d)
            if (moves_in(i, d)) r |= diag_step(b, d) & e;
        return r;
    }
    // does any piece of the mover have a hop?  (all pieces at once, per direction)
    __device__ __forceinline__ bool any_hop() const {
        const uint64_t e = empty(), o = opp();
        uint64_t r = 0;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const uint64_t movers = (side == 0) == (d < 2) ? own() : kings_own;
            r |= diag_step(diag_step(movers, d) & o, d) & e;
        }
        return r != 0;
    }
    __device__ __forceinline__ uint64_t movers() const { return pending >= 0 ? (1ull << pending) : own(); }
    __device__ __forceinline__ uint64_t dests(int i, bool cap) const { return cap ? hops_of(i) : steps_of(i); }
    // the position's legal-action count and capture mode, kept with the state
    // (the count is also the end test of the previous ply)
    // For one direction the destinations of different pieces are distinct
    // (each destination has one source cell), so the count is a popcount per
    // direction over all movers at once.
    __device__ __forceinline__ void refresh() {
        const uint64_t e = empty(), o = opp();
        uint64_t hop[4], step[4];
        bool cap = false;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const uint64_t fwd = (side == 0) == (d < 2);
            const uint64_t mv = pending >= 0 ? (1ull << pending) & (fwd ? own() : kings_own) : (fwd ? own() : kings_own);
            hop[d] = diag_step(diag_step(mv, d) & o, d) & e;
            step[d] = diag_step(mv, d) & e;
            cap = cap || hop[d] != 0;
        }
        capcache = pending >= 0 || cap;
        int n = 0;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const uint64_t dst = capcache ? hop[d] : step[d];
            n += __popcll(dst);
            // a destination minus the direction's step is its source
            const int back = (d == 0 ? 9 : d == 1 ? 7 : d == 2 ? -7 : -9) * (capcache ? 2 : 1);
            src[d] = back > 0 ? shl64c(dst, (uint32_t)back) : shr64c(dst, (uint32_t)-back);
        }
        ncache = outcome == kOngoing ? n : 0;
    }
    __device__ __forceinline__ bool capture_mode() const { return capcache; }
    __device__ __forceinline__ int count() const { return ncache; }
    __device__ __forceinline__ Mask legal() const { return ordinals64(ncache); }
    // The moves of piece i are the directions whose source set holds i
    // (ascending direction = ascending destination); every mover is counted
    // (no early exit) and the one holding the k-th move noted on the way.
    __device__ __forceinline__ void find(int k, int& from, int& to) const {
        int acc = 0, sel = -1, kk = 0;
        uint32_t dirs = 0;
        for (uint64_t m = movers(); m; m &= m - 1) {
            const int i = lowest(m);
            const uint32_t g = ((uint32_t)(src[0] >> i) & 1u) | (((uint32_t)(src[1] >> i) & 1u) << 1) |
                               (((uint32_t)(src[2] >> i) & 1u) << 2) | (((uint32_t)(src[3] >> i) & 1u) << 3);
            const int n = __popc(g);
            const bool hit = sel < 0 && k < acc + n;
            sel = hit ? i : sel;
            kk = hit ? k - acc : kk;
            dirs = hit ? g : dirs;
            acc += n;
        }
        from = sel;
        if (sel < 0) {
            to = -1;
            return;
        }
        const int d = select_bit(dirs, (uint32_t)kk);
        to = sel + (d == 0 ? -9 : d == 1 ? -7 : d == 2 ? 7 : 9) * (capture_mode() ? 2 : 1);
    }
    // The same lookup by the 32 lanes of a warp that all hold this position:
    // lane j reads the moves of the j-th mover (at most 12), a prefix sum over
    // the lanes finds the one holding move k.
    __device__ __forceinline__ void find_warp(int k, int& from, int& to, int lane) const {
        const uint64_t mv = movers();
        const int np = __popcll(mv);
        int i = -1, c = 0;
        uint32_t g = 0;
        if (lane < np) {
            i = select_bit(mv, (uint32_t)lane);
            g = ((uint32_t)(src[0] >> i) & 1u) | (((uint32_t)(src[1] >> i) & 1u) << 1) |
                (((uint32_t)(src[2] >> i) & 1u) << 2) | (((uint32_t)(src[3] >> i) & 1u) << 3);
            c = __popc(g);
        }
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += v;
        }
        const bool hit = lane < np && k >= incl - c && k < incl;
        const int srcl = __ffs(__ballot_sync(0xFFFFFFFFu, hit)) - 1;
        int t = -1;
        if (hit) {
            const int d = select_bit(g, (uint32_t)(k - (incl - c)));
            t = i + (d == 0 ? -9 : d == 1 ? -7 : d == 2 ? 7 : 9) * (capture_mode() ? 2 : 1);
        }
        from = __shfl_sync(0xFFFFFFFFu, i, srcl < 0 ? 0 : srcl);
        to = __shfl_sync(0xFFFFFFFFu, t, srcl < 0 ? 0 : srcl);
    }
    __device__ __forceinline__ void place_warp(int k, int lane) {
        int f, t;
        find_warp(k, f, t, lane);
        apply(f, t);
    }
    __device__ __forceinline__ void place(int k) {
        int f, t;
        find(k, f, t);
        apply(f, t);
    }
    // move the mover's piece from cell f to t, then capture, crowning, the
    // extra turn and the end test
    __device__ __forceinline__ void apply(int f, int t) {
        const int p = side;
        const uint64_t fb = 1ull << f, tb = 1ull << t;
        const bool king = (kings_own >> f) & 1;
        if (king) kings_own ^= fb | tb;
        else men_own ^= fb | tb;
        const int dist = t > f ? t - f : f - t;
        const bool hop = dist == 14 || dist == 18;
        if (hop) {
            const uint64_t keep = ~(1ull << ((f + t) >> 1));
            men_opp &= keep;
            kings_opp &= keep;
        }
        if (!king && (p == 0 ? t < 8 : t >= 56)) {  // crowned on the far row
            men_own &= ~tb;
            kings_own |= tb;
        }
        ++ply;
        if (hop && hops_of(t)) {
            pending = t;  // the same player captures again with this piece
        } else {
            pending = -1;
            uint64_t x = men_own;
            men_own = men_opp;
            men_opp = x;
            x = kings_own;
            kings_own = kings_opp;
            kings_opp = x;
            side ^= 1;
        }
        refresh();
        if (ncache == 0) outcome = p + 1;
    }
    __device__ __forceinline__ void pass() {}
    __device__ __forceinline__ int canon_of(int k) const {
        int f, t;
        find(k, f, t);
        return f * kCells + t;
    }
    __device__ __forceinline__ int bit_of(int a) const {
        const int f = a / kCells, t = a % kCells;
        const uint64_t mv = movers();
        if (!((mv >> f) & 1)) return -1;
        const bool cap = capture_mode();
        int base = 0;
        for (uint64_t m = mv & ((1ull << f) - 1); m; m &= m - 1) base += __popcll(dests(lowest(m), cap));
        const uint64_t d = dests(f, cap);
        if (!((d >> t) & 1)) return -1;
        return base + __popcll(d & ((1ull << t) - 1));
    }
    template <class F>
    __device__ __forceinline__ void for_each_move(F&& fn) const {
        const bool cap = capture_mode();
        for (uint64_t m = movers(); m; m &= m - 1) {
            const int i = lowest(m);
            for (uint64_t d = dests(i, cap); d; d &= d - 1) fn(i * kCells + lowest(d));
        }
    }
    __device__ __forceinline__ uint64_t occupied() const { return own() | opp(); }
    __device__ __forceinline__ void clear() { men_own = kings_own = men_opp = kings_opp = 0; }
    __device__ __forceinline__ int cell_value(int i) const {  // 1 / 2 men, 3 / 4 kings of P1 / P2
        const int mine = side + 1, theirs = 2 - side;
        if ((men_own >> i) & 1) return mine;
        if ((men_opp >> i) & 1) return theirs;
        if ((kings_own >> i) & 1) return mine + 2;
        if ((kings_opp >> i) & 1) return theirs + 2;
        return 0;
    }
    __device__ __forceinline__ void set_cell(int i, int v) {  // side already set
        const uint64_t b = 1ull << i;
        if (v == 0) return;
        const bool mine = ((v - 1) & 1) == side, king = v >= 3;
        if (mine) (king ? kings_own : men_own) |= b;
        else (king ? kings_opp : men_opp) |= b;
    }
    __device__ __forceinline__ int extra() const { return pending + 1; }
    __device__ __forceinline__ void set_extra(int x) { pending = x - 1; }  // call refresh() once the position is complete
    __device__ __forceinline__ void planes_out(uint64_t* w) const {  // P1 men, P1 kings, P2 men, P2 kings
        w[0] = side == 0 ? men_own : men_opp;
        w[1] = side == 0 ? kings_own : kings_opp;
        w[2] = side == 0 ? men_opp : men_own;
        w[3] = side == 0 ? kings_opp : kings_own;
    }
    __device__ __forceinline__ void planes_in(const uint64_t* w) {  // side already set
        men_own = side == 0 ? w[0] : w[2];
        kings_own = side == 0 ? w[1] : w[3];
        men_opp = side == 0 ? w[2] : w[0];
        kings_opp = side == 0 ? w[3] : w[1];
    }
    static constexpr int kWords = 5;
    __device__ __forceinline__ void save(uint64_t* w) const {
        w[0] = men_own;
        w[1] = kings_own;
        w[2] = men_opp;
        w[3] = kings_opp;
        w[4] = pack_small(ply, pending + 1, side, outcome);
    }
    __device__ __forceinline__ void load(const uint64_t* w) {
        men_own = w[0];
        kings_own = w[1];
        men_opp = w[2];
        kings_opp = w[3];
        int x;
        unpack_small(w[4], ply, x, side, outcome);
        pending = x - 1;
        passes = 0;
        refresh();
    }
};
template <>
struct IsMove<Draughts> {
    static constexpr bool value = true;
};

// --------------------------------------------------- Dai Hasami Shogi --
// word w of the cells of rows r0..r1 of the 9x9 board in the stride-10 layout
__host__ __device__ constexpr uint64_t hasami_rows(int r0, int r1, int w) {
    uint64_t m = 0;
    for (int b = 0; b < 64; ++b) {
        const int i = w * 64 + b, r = i / 10, c = i % 10;
        if (r >= r0 && r <= r1 && r < 9 && c < 9) m |= 1ull << b;
    }
    return m;
}
constexpr uint64_t kHasamiRows01Lo = hasami_rows(0, 1, 0), kHasamiRows01Hi = hasami_rows(0, 1, 1);
constexpr uint64_t kHasamiRows78Lo = hasami_rows(7, 8, 0), kHasamiRows78Hi = hasami_rows(7, 8, 1);
constexpr uint64_t kHasamiRows06Lo = hasami_rows(0, 6, 0), kHasamiRows06Hi = hasami_rows(0, 6, 1);
constexpr uint64_t kHasamiRows28Lo = hasami_rows(2, 8, 0), kHasamiRows28Hi = hasami_rows(2, 8, 1);
// word w of the transposed layout (bit 10 * column + row) holding rows r0..r1
__host__ __device__ constexpr uint64_t hasami_cols(int r0, int r1, int w) {
    uint64_t m = 0;
    for (int b = 0; b < 64; ++b) {
        const int i = w * 64 + b, c = i / 10, r = i % 10;
        if (r >= r0 && r <= r1 && r < 9 && c < 9) m |= 1ull << b;
    }
    return m;
}
constexpr uint64_t kHasamiStartTLo = hasami_cols(0, 1, 0) | hasami_cols(7, 8, 0);
constexpr uint64_t kHasamiStartTHi = hasami_cols(0, 1, 1) | hasami_cols(7, 8, 1);

// 9x9 in two words with a row stride of 10 (the empty tenth column stops
// horizontal runs from wrapping).  P1 fills rows 7-8, P2 rows 0-1.  A piece
// slides any distance orthogonally over empty cells or hops one adjacent
// piece (either side) onto the empty cell beyond; runs of opposing pieces
// that the moved piece closes against another own piece are removed, and so
// is an opposing piece in a corner whose two neighbours become the mover's;
// five in a row (row or column) with none on the mover's starting rows wins.
struct HasamiShogi {
    static constexpr int kGame = 10, kRows = 9, kCols = 9, kCells = 81, kCap = 200, kPlanes = 4, kActions = 6561;
    static constexpr int kStride = 10;
    static constexpr bool kHasPass = false;
    static constexpr bool kOrdinal = true;  // legal() holds the ordinals 0 .. count() - 1
    using Mask = BitsW<5>;  // ordinals: at most 18 pieces x 16 destinations = 288 legal actions
    B128 own, opp;          // relative to the side to move
    B128 occT;              // occupied cells transposed (bit 10 * column + row): columns as 10-bit windows
    int side, ply, passes, outcome;
    int ncache;             // legal actions of the position (refresh(); also the end test of a ply)

    __device__ __forceinline__ static B128 valid() { return B128{grid_word(9, 9, 10, false, 0), grid_word(9, 9, 10, false, 1)}; }
    __device__ __forceinline__ void reset() {
        own = B128{kHasamiRows78Lo, kHasamiRows78Hi};  // P1 on rows 7-8
        opp = B128{kHasamiRows01Lo, kHasamiRows01Hi};  // P2 on rows 0-1
        occT = B128{kHasamiStartTLo, kHasamiStartTHi};
        side = ply = passes = 0;
        outcome = kOngoing;
        ncache = 54;                                   // 9 pieces x 5 slides up + 9 hops
    }
    // one orthogonal step (and two, four): 0 up, 1 down, 2 left, 3 right
    __device__ __forceinline__ static B128 ortho(B128 b, int d) {
        switch (d) {
        case 0: return shr<10>(b);
        case 1: return shl<10>(b);
        case 2: return shr<1>(b);
        default: return shl<1>(b);
        }
    }
    __device__ __forceinline__ static B128 ortho2(B128 b, int d) {
        switch (d) {
        case 0: return shr<20>(b);
        case 1: return shl<20>(b);
        case 2: return shr<2>(b);
        default: return shl<2>(b);
        }
    }
    __device__ __forceinline__ static B128 ortho4(B128 b, int d) {
        switch (d) {
        case 0: return shr<40>(b);
        case 1: return shl<40>(b);
        case 2: return shr<4>(b);
        default: return shl<4>(b);
        }
    }
    // destinations of the piece on internal cell i: slides (occluded fill
    // over the empty cells, Kogge-Stone) and hops over one adjacent piece
    __device__ __forceinline__ B128 dests(int i) const {
        const B128 b = bit128(i), occ = own | opp, e = valid() & ~occ;
        B128 r{0, 0};
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            B128 g = b, p = e;
            g = g | (p & ortho(g, d));
            p = p & ortho(p, d);
            g = g | (p & ortho2(g, d));
            p = p & ortho2(p, d);
            g = g | (p & ortho4(g, d));
            r = r | (ortho(g, d) & e);                  // the empty run, up to 8 cells
            r = r | (ortho(ortho(b, d) & occ, d) & e);  // hop the adjacent piece
        }
        return r;
    }
    // The legal-action count of the mover, for all pieces at once: along one
    // direction the slide destinations of different pieces are disjoint (an
    // empty cell has one nearest piece behind it), and so are the hop
    // destinations, so each direction is one occluded fill and two popcounts.
    __device__ __forceinline__ int count_all() const {
        const B128 occ = own | opp, e = valid() & ~occ;
        int n = 0;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            B128 g = own, p = e;
            g = g | (p & ortho(g, d));
            p = p & ortho(p, d);
            g = g | (p & ortho2(g, d));
            p = p & ortho2(p, d);
            g = g | (p & ortho4(g, d));
            n += (int)popc(ortho(g, d) & e);
            n += (int)popc(ortho(ortho(own, d) & occ, d) & e);
        }
        return n;
    }
    __device__ __forceinline__ static int transposed(int i) { return 10 * (i % 10) + i / 10; }
    __device__ __forceinline__ void refresh() {
        occT = B128{0, 0};
        for (int w = 0; w < 2; ++w)
            for (uint64_t m = w ? (own.hi | opp.hi) : (own.lo | opp.lo); m; m &= m - 1)
                occT = occT | bit128(transposed(64 * w + lowest(m)));
        ncache = outcome == kOngoing ? count_all() : 0;
    }
    __device__ __forceinline__ int count() const { return ncache; }
    __device__ __forceinline__ Mask legal() const { return ordinalsW<5>(count()); }
    // bits at..at+8 of b: one row of the board (at = 10 * row) or one column
    // of the transpose (at = 10 * column); one funnel shift of two 32-bit words
    __device__ __forceinline__ static uint32_t field9(B128 b, int at) {
        const uint32_t w0 = (uint32_t)b.lo, w1 = (uint32_t)(b.lo >> 32), w2 = (uint32_t)b.hi, w3 = (uint32_t)(b.hi >> 32);
        const int q = at >> 5;
        const uint32_t x = q == 0 ? w0 : (q == 1 ? w1 : w2), y = q == 0 ? w1 : (q == 1 ? w2 : w3);
        return __funnelshift_r(x, y, (uint32_t)at & 31u) & 0x1FFu;
    }
    // the blocked cells of a row or column as a window: cell j at bit j + 2,
    // and two set bits past each end (the edge stops runs and hops as a
    // piece does)
    __device__ __forceinline__ static uint32_t window(B128 occ, int at) { return (field9(occ, at) << 2) | 0x1803u; }
    // The moves of one piece without forming its destination set: in the
    // window of its row (column) the slide to the right (down) is the run of
    // clear bits above it and to the left (up) the run below it; a hop needs
    // the adjacent cell blocked by a piece and the cell beyond it clear.
    struct Runs {
        int up, left, right, down;
        int hup, hleft, hright, hdown;
        __device__ __forceinline__ int total() const { return up + left + right + down + hup + hleft + hright + hdown; }
    };
    __device__ __forceinline__ static void axis(uint32_t w, int j, int& lo, int& hi, int& hlo, int& hhi) {
        const uint32_t a = w >> (j + 3);                        // bit 0: the cell after j
        hi = __ffs(a) - 1;
        lo = j - 30 + __clz(w & ((1u << (j + 2)) - 1u));        // nearest blocked bit below j
        hhi = (int)(a & ~(a >> 1) & 1u);
        hlo = (int)((w >> (j + 1)) & ~(w >> j) & 1u);
    }
    __device__ __forceinline__ static Runs runs_of(uint32_t row, uint32_t col, int r, int c) {
        Runs x;
        axis(row, c, x.left, x.right, x.hleft, x.hright);
        axis(col, r, x.up, x.down, x.hup, x.hdown);
        return x;
    }
    // the k-th destination of piece i in ascending cell order: cells above
    // it, then left of it, right of it, below it
    __device__ __forceinline__ static int dest_of(int i, const Runs& x, int k) {
        const int nu = x.up + x.hup, nl = x.left + x.hleft, nr = x.right + x.hright;
        if (k < nu) return x.hup ? i - 20 : i - 10 * (x.up - k);
        k -= nu;
        if (k < nl) return x.hleft ? i - 2 : i - (x.left - k);
        k -= nl;
        if (k < nr) return x.hright ? i + 2 : i + 1 + k;
        k -= nr;
        return x.hdown ? i + 20 : i + 10 * (1 + k);
    }
    __device__ __forceinline__ Runs runs_at(B128 occ, int i) const {
        const int r = i / 10, c = i - 10 * r;
        return runs_of(window(occ, 10 * r), window(occT, 10 * c), r, c);
    }
    // Every piece is counted (no early exit): the counts do not depend on k,
    // so their latencies overlap, and the piece holding the k-th move is
    // noted on the way.
    __device__ __forceinline__ void find(int k, int& from, int& to) const {
        const B128 occ = own | opp;
        int acc = 0, sel = -1, kk = 0;
        for (int w = 0; w < 2; ++w) {
            for (uint64_t m = w ? own.hi : own.lo; m; m &= m - 1) {
                const int i = 64 * w + lowest(m);
                const int n = runs_at(occ, i).total();
                const bool hit = sel < 0 && k < acc + n;
                sel = hit ? i : sel;
                kk = hit ? k - acc : kk;
                acc += n;
            }
        }
        from = sel;
        to = sel < 0 ? -1 : dest_of(sel, runs_at(occ, sel), kk);
    }
    // The same lookup by the 32 lanes of a warp that all hold this position:
    // lane j counts the moves of the j-th piece (at most 18), a prefix sum
    // over the lanes finds the piece holding move k, and its lane forms the
    // destination.
    __device__ __forceinline__ void find_warp(int k, int& from, int& to, int lane) const {
        const B128 occ = own | opp;
        const int np = (int)popc(own);
        int i = -1, c = 0;
        Runs x{};
        if (lane < np) {
            i = select_bit(own, (uint32_t)lane);
            x = runs_at(occ, i);
            c = x.total();
        }
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += v;
        }
        const bool hit = lane < np && k >= incl - c && k < incl;
        const int src = __ffs(__ballot_sync(0xFFFFFFFFu, hit)) - 1;
        const int t = hit ? dest_of(i, x, k - (incl - c)) : -1;
        from = __shfl_sync(0xFFFFFFFFu, i, src < 0 ? 0 : src);
        to = __shfl_sync(0xFFFFFFFFu, t, src < 0 ? 0 : src);
    }
    __device__ __forceinline__ void place_warp(int k, int lane) {
        int f, t;
        find_warp(k, f, t, lane);
        apply(f, t);
    }
    __device__ __forceinline__ bool five() const {  // the mover, outside its starting rows
        const B128 m = own & (side == 0 ? B128{kHasamiRows06Lo, kHasamiRows06Hi} : B128{kHasamiRows28Lo, kHasamiRows28Hi});
        const B128 h = m & shr<1>(m) & shr<2>(m) & shr<3>(m) & shr<4>(m);
        const B128 v = m & shr<10>(m) & shr<20>(m) & shr<30>(m) & shr<40>(m);
        return any(h | v);
    }
    __device__ __forceinline__ void place(int k) {
        int f, t;
        find(k, f, t);
        apply(f, t);
    }
    // move the mover's piece from internal cell f to t, then captures and end test
    __device__ __forceinline__ void apply(int f, int t) {
        const int p = side;
        const B128 tb = bit128(t), tT = bit128(transposed(t));
        own = (own & ~bit128(f)) | tb;
        occT = (occT & ~bit128(transposed(f))) | tT;
        // custodial captures along the four directions from the moved piece
        // (walked in both layouts: a row of the board is a column of the transpose)
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const int dT = d ^ 2;
            B128 run{0, 0}, runT{0, 0}, x = ortho(tb, d), xT = ortho(tT, dT);
            for (int s = 0; s < 8 && any(x & opp); ++s) {
                run = run | x;
                runT = runT | xT;
                x = ortho(x, d);
                xT = ortho(xT, dT);
            }
            if (any(x & own)) {
                opp = opp & ~run;
                occT = occT & ~runT;
            }
        }
        // corner captures: an opposing corner piece whose two neighbours are
        // now the mover's, one of them the moved piece
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int corner = c == 0 ? 0 : (c == 1 ? 8 : (c == 2 ? 80 : 88));
            const int n1 = c == 0 ? 10 : (c == 1 ? 18 : (c == 2 ? 70 : 78));
            const int n2 = c == 0 ? 1 : (c == 1 ? 7 : (c == 2 ? 81 : 87));
            if (any(opp & bit128(corner)) && any(own & bit128(n1)) && any(own & bit128(n2)) && (t == n1 || t == n2)) {
                opp = opp & ~bit128(corner);
                occT = occT & ~bit128(c == 0 ? 0 : (c == 1 ? 80 : (c == 2 ? 8 : 88)));
            }
        }
        const bool won = five();
        const B128 x = own;
        own = opp;
        opp = x;
        ++ply;
        side ^= 1;
        ncache = count_all();  // the next player's legal actions
        if (won || ncache == 0) outcome = p + 1;
    }
    __device__ __forceinline__ void pass() {}
    __device__ __forceinline__ static int canon_cell(int b) { return (b / kStride) * kCols + b % kStride; }
    __device__ __forceinline__ static int internal_cell(int c) { return (c / kCols) * kStride + c % kCols; }
    __device__ __forceinline__ int canon_of(int k) const {
        int f, t;
        find(k, f, t);
        return canon_cell(f) * kCells + canon_cell(t);
    }
    __device__ __forceinline__ static B128 below(int t) {  // bits 0 .. t-1
        return t < 64 ? B128{(1ull << t) - 1, 0ull} : B128{~0ull, t == 64 ? 0ull : ((1ull << (t - 64)) - 1)};
    }
    __device__ __forceinline__ int bit_of(int a) const {
        const int f = internal_cell(a / kCells), t = internal_cell(a % kCells);
        if (!any(own & bit128(f))) return -1;
        int base = 0;
        const B128 before = own & below(f);
        for (uint64_t m = before.lo; m; m &= m - 1) base += (int)popc(dests(lowest(m)));
        for (uint64_t m = before.hi; m; m &= m - 1) base += (int)popc(dests(64 + lowest(m)));
        const B128 d = dests(f);
        if (!any(d & bit128(t))) return -1;
        return base + (int)popc(d & below(t));
    }
    template <class F>
    __device__ __forceinline__ void for_each_move(F&& fn) const {
        for (int w = 0; w < 2; ++w)
            for (uint64_t m = w ? own.hi : own.lo; m; m &= m - 1) {
                const int i = 64 * w + lowest(m);
                const B128 d = dests(i);
                for (uint64_t q = d.lo; q; q &= q - 1) fn(canon_cell(i) * kCells + canon_cell(lowest(q)));
                for (uint64_t q = d.hi; q; q &= q - 1) fn(canon_cell(i) * kCells + canon_cell(64 + lowest(q)));
            }
    }
    __device__ __forceinline__ B128 occupied() const { return own | opp; }
    __device__ __forceinline__ void clear() { own = opp = B128{0, 0}; }
    __device__ __forceinline__ int cell_value(int c) const {
        const B128 b = bit128(internal_cell(c));
        return any(own & b) ? side + 1 : (any(opp & b) ? 2 - side : 0);
    }
    __device__ __forceinline__ void set_cell(int c, int v) {  // side already set
        if (v == 0) return;
        const B128 b = bit128(internal_cell(c));
        if (v - 1 == side) own = own | b;
        else opp = opp | b;
    }
    __device__ __forceinline__ int extra() const { return 0; }
    __device__ __forceinline__ void set_extra(int) {}
    __device__ __forceinline__ void planes_out(uint64_t* w) const {  // P1 lo, hi, P2 lo, hi
        const B128 a = side == 0 ? own : opp, b = side == 0 ? opp : own;
        w[0] = a.lo;
        w[1] = a.hi;
        w[2] = b.lo;
        w[3] = b.hi;
    }
    __device__ __forceinline__ void planes_in(const uint64_t* w) {  // side already set
        const B128 a{w[0], w[1]}, b{w[2], w[3]};
        own = side == 0 ? a : b;
        opp = side == 0 ? b : a;
    }
    static constexpr int kWords = 7;
    __device__ __forceinline__ void save(uint64_t* w) const {
        w[0] = own.lo;
        w[1] = own.hi;
        w[2] = opp.lo;
        w[3] = opp.hi;
        w[4] = pack_small(ply, passes, side, outcome);
        w[5] = occT.lo;
        w[6] = occT.hi;
    }
    __device__ __forceinline__ void load(const uint64_t* w) {
        own = B128{w[0], w[1]};
        opp = B128{w[2], w[3]};
        unpack_small(w[4], ply, passes, side, outcome);
        occT = B128{w[5], w[6]};
        ncache = outcome == kOngoing ? count_all() : 0;
    }
};
template <>
struct IsMove<HasamiShogi> {
    static constexpr bool value = true;
};

}  // namespace ludax
