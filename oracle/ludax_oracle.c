/*
 * ludax_oracle.c -- plain, slow CPU oracle for the Ludax board-game hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA path under paper_2506_22609_b300/csrc.
 *
 * What it computes (Ludax, arXiv 2506.22609):
 *   - the rules of Tic-Tac-Toe, Connect Four, Hex and Reversi/Othello as the
 *     paper's game appendix states them (App. C, "Benchmark Game
 *     Descriptions"), over a row-major int8 cell array with row 0 at the top
 *     (cell numbering as in the English Draughts listing of App. A, where P1
 *     moves "up" and starts on cells 40..62);
 *   - the action = destination-cell convention of Sec. 3.4 (Connect Four's
 *     legal cells are the empty cells directly above an occupied cell or on
 *     the bottom row), plus one pass action for Reversi (force_pass, App. B);
 *   - ordered end rules, a win checked before a draw (Sec. 3.3);
 *   - uniform-random playouts (the random-policy benchmark of Sec. 6) driven
 *     by a counter-based splitmix64 keyed on (seed, env, ply).
 *
 * Every check is a direct scan of the cell array: lines are found by testing
 * every start cell and direction, Reversi legality and flips walk each ray
 * cell by cell, and Hex connectivity is a breadth-first search from the
 * mover's first edge.  No bitboards, no incremental state.
 *
 * The line-game family (App. C): Gomoku 15x15 (a line of exactly five wins,
 * six or more does not), Pente 19x19 (five or more in a row wins; placing a
 * stone that closes own-opp-opp-own along any of 8 directions removes the two
 * opponent stones; ten captured stones win; P1's first move is the centre),
 * Yavalath on the 61-cell hexagon (four in a row wins, otherwise three in a
 * row loses); all three end in a draw on a full board.  The parametric line
 * game (place on an empty cell, optionally with Connect-Four gravity; a line
 * of at least -- or exactly -- L wins, or loses in the misere variant; a full
 * board draws) covers Tic-Tac-Toe, Connect Four and their variants on any
 * board of up to 128 padded cells.
 *
 * Readings where the paper is silent:
 *   Hex neighbours of (r,c): (r-1,c) (r+1,c) (r,c-1) (r,c+1) (r-1,c+1) (r+1,c-1);
 *   Reversi: P1 = black moves first; white on D4,E5 = cells 27,36, black on
 *   D5,E4 = cells 35,28 (algebraic rows counted from the top); a pass is the
 *   action id 64, legal only when no cell is; two consecutive passes end the
 *   game; a tie in disc count is a draw;
 *   an illegal action ends the game: the mover loses (reward -1, opponent +1);
 *   ply caps 9 / 42 / 128 / n*n mark an env CAPPED (never reached by a correct
 *   implementation of these games).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_TTT 0
#define OR_C4 1
#define OR_OTHELLO 2
#define OR_HEX 3
#define OR_GOMOKU 4
#define OR_PENTE 5
#define OR_YAVALATH 6
#define OR_LINE 7 /* parametric line game; the game argument packs 7 | L << 8 | flags << 12 */
#define OR_WOLF 8     /* Wolf and Sheep, 8x8 */
#define OR_DRAUGHTS 9 /* English Draughts, 8x8 */
#define OR_HASAMI 10  /* Dai Hasami Shogi, 9x9 */
#define OR_LINE_EXACT 1
#define OR_LINE_GRAVITY 2
#define OR_LINE_MISERE 4

#define OR_ONGOING (-1)
#define OR_DRAW 0
#define OR_P1 1
#define OR_P2 2
#define OR_CAPPED 3

#define OR_MAXCELLS 512
#define OR_MAXACTIONS (81 * 81 + 1) /* move games: action = from * cells + to */

typedef struct {
    int32_t game, rows, cols, ncells;
    int8_t cell[OR_MAXCELLS]; /* 0 empty, 1 P1, 2 P2; index r*cols + c, r = 0 top
                                 (Yavalath: row-major over the 61 cells of the hexagon) */
    int32_t to_move;          /* 1 or 2 */
    int32_t ply;              /* plies played so far, passes included */
    int32_t passes;           /* consecutive passes (Reversi) */
    int32_t outcome;          /* OR_ONGOING, OR_DRAW, OR_P1, OR_P2, OR_CAPPED */
    int32_t illegal;          /* 1 when the game ended on an illegal action */
    int32_t captures[3];      /* Pente: opponent stones captured by player 1 / 2 */
    int32_t line, flags;      /* parametric line game: line length, OR_LINE_* flags */
    int32_t pending;          /* Draughts: cell of the piece that must capture again, -1 if none */
} ogame;

/* ------------------------------------------------------------------ RNG --
 * splitmix64 (Steele, Lea and Flood, OOPSLA 2014; the form published by
 * Vigna): add the golden-ratio increment, then the finaliser
 * z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27; z *= 0x94D049BB133111EB;
 * z ^= z>>31.  oracle_sm(x) is one output for the state x.                  */
uint64_t oracle_sm(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* The counter-based draw for one ply of one env: the key of an env is
 * sm(sm(seed) ^ env) with env the global env index; the draw for a ply is
 * sm(key ^ ply).                                                           */
uint64_t oracle_draw(uint64_t seed, uint64_t env, uint64_t ply) {
    uint64_t key = oracle_sm(oracle_sm(seed) ^ env);
    return oracle_sm(key ^ ply);
}

/* Uniform index in [0, n) from the top 32 bits of a draw (multiply-shift). */
uint32_t oracle_pick(uint64_t r, uint32_t n) {
    uint64_t hi = r >> 32;
    return (uint32_t)((hi * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------ geometry -- */
/* Yavalath's hexagon (side 5, 61 cells, the long diagonal drawn left to
 * right) in axial coordinates: rows r = 0..8, columns c = 0..8 with
 * |r - c| <= 4; neighbours differ by (0,+-1), (+-1,0) or (+-1,+-1).  Cells are
 * numbered row by row, left to right. */
static int yav_valid(int r, int c) { return r >= 0 && r < 9 && c >= 0 && c < 9 && (r - c <= 4) && (c - r <= 4); }
static int yav_id(int r, int c) {
    int id = 0;
    for (int rr = 0; rr < r; ++rr) id += 9 - (rr > 4 ? rr - 4 : 4 - rr);
    return id + c - (r > 4 ? r - 4 : 0);
}
static void yav_rc(int id, int* r, int* c) {
    int rr = 0;
    for (;;) {
        int len = 9 - (rr > 4 ? rr - 4 : 4 - rr);
        if (id < len) break;
        id -= len;
        rr++;
    }
    *r = rr;
    *c = id + (rr > 4 ? rr - 4 : 0);
}

/* canonical id of (r, c), or -1 off the board */
static int cell_id(const ogame* g, int r, int c) {
    if (g->game == OR_YAVALATH) return yav_valid(r, c) ? yav_id(r, c) : -1;
    return (r >= 0 && r < g->rows && c >= 0 && c < g->cols) ? r * g->cols + c : -1;
}
static void cell_rc(const ogame* g, int id, int* r, int* c) {
    if (g->game == OR_YAVALATH) yav_rc(id, r, c);
    else { *r = id / g->cols; *c = id % g->cols; }
}
static int in_board(const ogame* g, int r, int c) { return cell_id(g, r, c) >= 0; }
static int at(const ogame* g, int r, int c) { return g->cell[cell_id(g, r, c)]; }

int oracle_ply_cap(int game, int rows, int cols) {
    switch (game & 0xFF) {
    case OR_LINE: return rows * cols;
    case OR_TTT: return 9;
    case OR_C4: return 42;
    case OR_OTHELLO: return 128;
    case OR_HEX: return rows * cols;
    case OR_GOMOKU: return rows * cols;
    case OR_PENTE: return 2000;
    case OR_YAVALATH: return 61;
    case OR_WOLF:
    case OR_DRAUGHTS:
    case OR_HASAMI: return 200; /* Sec. 6: unbounded games stop after 200 turns */
    }
    return 0;
}

/* Number of actions: one per cell, plus the pass for Reversi. */
int oracle_num_cells(int game, int rows, int cols) { return (game & 0xFF) == OR_YAVALATH ? 61 : rows * cols; }

static int is_move_game(int game) { return game == OR_WOLF || game == OR_DRAUGHTS || game == OR_HASAMI; }

int oracle_num_actions(int game, int rows, int cols) {
    int n = oracle_num_cells(game, rows, cols);
    if (is_move_game(game)) return n * n; /* action = from * cells + to */
    return n + (game == OR_OTHELLO ? 1 : 0);
}

int oracle_check_params(int game, int rows, int cols) {
    if ((game & 0xFF) == OR_LINE) {
        int L = (game >> 8) & 15, fl = (game >> 12) & 7;
        if (game >> 15) return -1;
        (void)fl;
        return (rows >= 1 && cols >= 1 && rows * (cols + 1) <= 128 && L >= 2 && L <= (rows > cols ? rows : cols)) ? 0
                                                                                                               : -1;
    }
    switch (game) {
    case OR_TTT: return (rows == 3 && cols == 3) ? 0 : -1;
    case OR_C4: return (rows == 6 && cols == 7) ? 0 : -1;
    case OR_OTHELLO: return (rows == 8 && cols == 8) ? 0 : -1;
    case OR_HEX: return (rows == cols && rows >= 2 && rows <= 11) ? 0 : -1;
    case OR_GOMOKU: return (rows == 15 && cols == 15) ? 0 : -1;
    case OR_PENTE: return (rows == 19 && cols == 19) ? 0 : -1;
    case OR_YAVALATH: return (rows == 9 && cols == 9) ? 0 : -1;
    case OR_WOLF:
    case OR_DRAUGHTS: return (rows == 8 && cols == 8) ? 0 : -1;
    case OR_HASAMI: return (rows == 9 && cols == 9) ? 0 : -1;
    }
    return -1;
}

/* Start position: an empty board, except Reversi's four discs. */
int oracle_init(ogame* g, int game, int rows, int cols) {
    if (oracle_check_params(game, rows, cols) != 0) return -1;
    memset(g, 0, sizeof(*g));
    if ((game & 0xFF) == OR_LINE) {
        g->line = (game >> 8) & 15;
        g->flags = (game >> 12) & 7;
        game = OR_LINE;
    }
    g->game = game;
    g->rows = rows;
    g->cols = cols;
    g->ncells = oracle_num_cells(game, rows, cols);
    g->to_move = 1;
    g->outcome = OR_ONGOING;
    g->pending = -1;
    if (game == OR_WOLF) {
        /* four sheep (P1) on the dark cells of the bottom row, the wolf (P2)
         * on the left one of the two central dark cells of the top row */
        for (int c = 0; c < 8; c += 2) g->cell[7 * 8 + c] = 1;
        g->cell[3] = 2;
    }
    if (game == OR_DRAUGHTS) {
        /* men on the dark cells ((r + c) odd): P1 on rows 5-7, P2 on rows 0-2 */
        for (int r = 0; r < 8; r++)
            for (int c = 0; c < 8; c++)
                if ((r + c) % 2 == 1 && (r >= 5 || r <= 2)) g->cell[r * 8 + c] = (int8_t)(r >= 5 ? 1 : 2);
    }
    if (game == OR_HASAMI) {
        /* P1 fills the bottom two rows, P2 the top two */
        for (int c = 0; c < 9; c++) {
            g->cell[0 * 9 + c] = g->cell[1 * 9 + c] = 2;
            g->cell[7 * 9 + c] = g->cell[8 * 9 + c] = 1;
        }
    }
    if (game == OR_OTHELLO) {
        /* D4 and E5 white (P2); D5 and E4 black (P1); row 4 is index 3. */
        g->cell[3 * 8 + 3] = 2; /* D4 = 27 */
        g->cell[4 * 8 + 4] = 2; /* E5 = 36 */
        g->cell[4 * 8 + 3] = 1; /* D5 = 35 */
        g->cell[3 * 8 + 4] = 1; /* E4 = 28 */
    }
    return 0;
}

/* ---------------------------------------------------------------- lines --
 * Does player p own L consecutive cells along any row, column or diagonal?
 * Every start cell and every one of the four directions is tested.        */
static int has_line(const ogame* g, int p, int L) {
    static const int dr[4] = {0, 1, 1, 1};
    static const int dc[4] = {1, 0, 1, -1};
    int nd = g->game == OR_YAVALATH ? 3 : 4; /* the hexagon's three axes: (0,1) (1,0) (1,1) */
    for (int r = 0; r < g->rows; r++)
        for (int c = 0; c < g->cols; c++)
            for (int d = 0; d < nd; d++) {
                int k = 0;
                while (k < L && in_board(g, r + k * dr[d], c + k * dc[d]) &&
                       at(g, r + k * dr[d], c + k * dc[d]) == p)
                    k++;
                if (k == L) return 1;
            }
    return 0;
}

/* Does player p own a maximal run of exactly L cells in a row (the cells
 * just before and just after the run are not p's)? */
static int has_line_exact(const ogame* g, int p, int L) {
    static const int dr[4] = {0, 1, 1, 1};
    static const int dc[4] = {1, 0, 1, -1};
    for (int r = 0; r < g->rows; r++)
        for (int c = 0; c < g->cols; c++)
            for (int d = 0; d < 4; d++) {
                int pr = r - dr[d], pc = c - dc[d];
                if (in_board(g, pr, pc) && at(g, pr, pc) == p) continue; /* not the start of a run */
                int k = 0;
                while (in_board(g, r + k * dr[d], c + k * dc[d]) && at(g, r + k * dr[d], c + k * dc[d]) == p) k++;
                if (k == L) return 1;
            }
    return 0;
}

static int board_full(const ogame* g) {
    for (int i = 0; i < g->ncells; i++)
        if (g->cell[i] == 0) return 0;
    return 1;
}

/* ------------------------------------------------------------- Reversi -- */
static const int ODR[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
static const int ODC[8] = {-1, 0, 1, -1, 1, -1, 0, 1};

/* Length of the run of opponent discs starting next to (r,c) in direction d
 * that is closed by one of p's discs; 0 if there is no such custodial run. */
static int custodial_run(const ogame* g, int p, int r, int c, int d) {
    int q = 3 - p, k = 1;
    while (in_board(g, r + k * ODR[d], c + k * ODC[d]) && at(g, r + k * ODR[d], c + k * ODC[d]) == q)
        k++;
    if (k == 1) return 0;
    if (!in_board(g, r + k * ODR[d], c + k * ODC[d])) return 0;
    return at(g, r + k * ODR[d], c + k * ODC[d]) == p ? k - 1 : 0;
}

static int othello_cell_legal(const ogame* g, int p, int i) {
    int r = i / g->cols, c = i % g->cols;
    if (g->cell[i] != 0) return 0;
    for (int d = 0; d < 8; d++)
        if (custodial_run(g, p, r, c, d) > 0) return 1;
    return 0;
}

/* ----------------------------------------------------------------- Hex --
 * Breadth-first search over p's stones from p's first edge; p connects
 * when the search reaches p's second edge.  P1 joins row 0 to row n-1,
 * P2 joins column 0 to column n-1.                                       */
static const int HDR[6] = {-1, 1, 0, 0, -1, 1};
static const int HDC[6] = {0, 0, -1, 1, 1, -1};

static int hex_connects(const ogame* g, int p) {
    int n = g->rows;
    int seen[OR_MAXCELLS];
    int queue[OR_MAXCELLS];
    int head = 0, tail = 0;
    memset(seen, 0, sizeof(seen));
    for (int t = 0; t < n; t++) {
        int r = (p == 1) ? 0 : t;
        int c = (p == 1) ? t : 0;
        int i = r * n + c;
        if (g->cell[i] == p) {
            seen[i] = 1;
            queue[tail++] = i;
        }
    }
    while (head < tail) {
        int i = queue[head++];
        int r = i / n, c = i % n;
        if ((p == 1 && r == n - 1) || (p == 2 && c == n - 1)) return 1;
        for (int d = 0; d < 6; d++) {
            int rr = r + HDR[d], cc = c + HDC[d];
            if (!in_board(g, rr, cc)) continue;
            int j = rr * n + cc;
            if (!seen[j] && g->cell[j] == p) {
                seen[j] = 1;
                queue[tail++] = j;
            }
        }
    }
    return 0;
}

/* For a full or partial Hex board: bit 0 set if P1 connects, bit 1 if P2. */
int oracle_hex_connections(int n, const int8_t* cells) {
    ogame g;
    if (oracle_init(&g, OR_HEX, n, n) != 0) return -1;
    memcpy(g.cell, cells, (size_t)(n * n));
    return (hex_connects(&g, 1) ? 1 : 0) | (hex_connects(&g, 2) ? 2 : 0);
}

/* ---------------------------------------------------------- move games --
 * Wolf and Sheep, English Draughts, Dai Hasami Shogi (App. C): pieces move
 * from one cell to another, so an action is from * cells + to.  Cell values:
 * 1 / 2 a piece of P1 / P2; 3 / 4 a king of P1 / P2 (Draughts).  P1 starts at
 * the bottom and its "forward" is up (row 0 is the top).
 *   Wolf and Sheep: sheep (P1) step diagonally forward, the wolf (P2)
 *   diagonally in any direction, always onto an empty cell; the wolf wins on
 *   reaching the bottom row.
 *   Draughts: men step diagonally forward onto an empty cell or hop over an
 *   adjacent opposing piece diagonally forward onto the empty cell beyond,
 *   removing it; kings do both in all four diagonal directions; when any hop
 *   exists, only hops are legal; a man ending on the far row becomes a king;
 *   after a hop, if the moved piece (promoted or not) can hop again, the same
 *   player moves again and only that piece's hops are legal.
 *   Dai Hasami Shogi: a piece slides any distance orthogonally over empty
 *   cells, or hops orthogonally over one adjacent piece of either side onto
 *   the empty cell beyond (no capture); after the move, every straight
 *   orthogonal run of opposing pieces that starts next to the moved piece and
 *   ends at another piece of the mover is removed, and an opposing piece in a
 *   corner whose two orthogonal neighbours are then both the mover's, one of
 *   them the moved piece, is removed; five or more in a row, horizontally or
 *   vertically, with none of the five on the mover's two starting rows, wins.
 * In all three, the mover also wins when the player to move next has no
 * legal action (as the Draughts listing of App. A ends its games). */
static void finish(ogame* g, int outcome);

static int owner_of(int v) { return v == 0 ? 0 : ((v == 1 || v == 3) ? 1 : 2); }

static int on_board(const ogame* g, int r, int c) { return r >= 0 && r < g->rows && c >= 0 && c < g->cols; }

static int cell_at(const ogame* g, int r, int c) { return g->cell[r * g->cols + c]; }

/* the diagonal directions a Draughts piece of value v moves in */
static int draughts_dirs(int v, int dr[4], int dc[4]) {
    int n = 0, king = v >= 3, p = owner_of(v);
    for (int sr = -1; sr <= 1; sr += 2)
        for (int sc = -1; sc <= 1; sc += 2)
            if (king || (p == 1 && sr == -1) || (p == 2 && sr == 1)) {
                dr[n] = sr;
                dc[n] = sc;
                n++;
            }
    return n;
}

/* hops of the Draughts piece on cell i into legal[] (NULL: count only) */
static int draughts_hops(const ogame* g, int i, uint8_t* legal) {
    int dr[4], dc[4], r = i / 8, c = i % 8, v = g->cell[i], p = owner_of(v), n = 0;
    int k = draughts_dirs(v, dr, dc);
    for (int d = 0; d < k; d++) {
        int r1 = r + dr[d], c1 = c + dc[d], r2 = r + 2 * dr[d], c2 = c + 2 * dc[d];
        if (on_board(g, r2, c2) && owner_of(cell_at(g, r1, c1)) == 3 - p && cell_at(g, r2, c2) == 0) {
            if (legal) legal[i * 64 + r2 * 8 + c2] = 1;
            n++;
        }
    }
    return n;
}

static int move_legal(const ogame* g, int p, uint8_t* legal) {
    int N = g->ncells, n = 0;
    if (legal) memset(legal, 0, (size_t)N * N);
    if (g->game == OR_WOLF) {
        for (int i = 0; i < N; i++) {
            int r = i / 8, c = i % 8;
            if (g->cell[i] != p) continue;
            for (int sr = -1; sr <= 1; sr += 2)
                for (int sc = -1; sc <= 1; sc += 2) {
                    if (p == 1 && sr == 1) continue; /* sheep only go forward (up) */
                    if (on_board(g, r + sr, c + sc) && cell_at(g, r + sr, c + sc) == 0) {
                        if (legal) legal[i * N + (r + sr) * 8 + c + sc] = 1;
                        n++;
                    }
                }
        }
        return n;
    }
    if (g->game == OR_DRAUGHTS) {
        if (g->pending >= 0) return draughts_hops(g, g->pending, legal);
        for (int i = 0; i < N; i++)
            if (owner_of(g->cell[i]) == p) n += draughts_hops(g, i, legal);
        if (n > 0) return n; /* captures take priority over steps */
        for (int i = 0; i < N; i++) {
            int dr[4], dc[4], r = i / 8, c = i % 8, k;
            if (owner_of(g->cell[i]) != p) continue;
            k = draughts_dirs(g->cell[i], dr, dc);
            for (int d = 0; d < k; d++)
                if (on_board(g, r + dr[d], c + dc[d]) && cell_at(g, r + dr[d], c + dc[d]) == 0) {
                    if (legal) legal[i * N + (r + dr[d]) * 8 + c + dc[d]] = 1;
                    n++;
                }
        }
        return n;
    }
    /* Dai Hasami Shogi */
    for (int i = 0; i < N; i++) {
        static const int DR[4] = {-1, 1, 0, 0}, DC[4] = {0, 0, -1, 1};
        int r = i / 9, c = i % 9;
        if (g->cell[i] != p) continue;
        for (int d = 0; d < 4; d++) {
            int k = 1;
            while (on_board(g, r + k * DR[d], c + k * DC[d]) && cell_at(g, r + k * DR[d], c + k * DC[d]) == 0) {
                if (legal) legal[i * N + (r + k * DR[d]) * 9 + c + k * DC[d]] = 1;
                n++;
                k++;
            }
            if (k == 1 && on_board(g, r + 2 * DR[d], c + 2 * DC[d]) && cell_at(g, r + 2 * DR[d], c + 2 * DC[d]) == 0) {
                if (legal) legal[i * N + (r + 2 * DR[d]) * 9 + c + 2 * DC[d]] = 1; /* hop the adjacent piece */
                n++;
            }
        }
    }
    return n;
}

/* Hasami: does p own five in a row (row or column) outside its two starting rows? */
static int hasami_line(const ogame* g, int p) {
    int lo = p == 1 ? 0 : 2, hi = p == 1 ? 6 : 8; /* rows that count */
    for (int r = lo; r <= hi; r++)
        for (int c = 0; c < 9; c++) {
            int h = 0, v = 0;
            for (int k = 0; k < 5; k++) {
                h += c + k < 9 && cell_at(g, r, c + k) == p;
                v += r + k <= hi && cell_at(g, r + k, c) == p;
            }
            if (h == 5 || v == 5) return 1;
        }
    return 0;
}

static void move_apply(ogame* g, int action) {
    int N = g->ncells, from = action / N, to = action % N, p = g->to_move, v = g->cell[from];
    int rf = from / g->cols, cf = from % g->cols, rt = to / g->cols, ct = to % g->cols, again = 0;
    g->cell[from] = 0;
    g->cell[to] = (int8_t)v;
    if (g->game == OR_DRAUGHTS) {
        int hop = rt - rf == 2 || rf - rt == 2;
        if (hop) g->cell[((rf + rt) / 2) * 8 + (cf + ct) / 2] = 0;
        if (v < 3 && ((p == 1 && rt == 0) || (p == 2 && rt == 7))) g->cell[to] = (int8_t)(v + 2);
        again = hop && draughts_hops(g, to, NULL) > 0;
        g->pending = again ? to : -1;
    }
    if (g->game == OR_HASAMI) {
        static const int DR[4] = {-1, 1, 0, 0}, DC[4] = {0, 0, -1, 1};
        for (int d = 0; d < 4; d++) {
            int k = 1;
            while (on_board(g, rt + k * DR[d], ct + k * DC[d]) && cell_at(g, rt + k * DR[d], ct + k * DC[d]) == 3 - p) k++;
            if (k > 1 && on_board(g, rt + k * DR[d], ct + k * DC[d]) && cell_at(g, rt + k * DR[d], ct + k * DC[d]) == p)
                for (int j = 1; j < k; j++) g->cell[(rt + j * DR[d]) * 9 + ct + j * DC[d]] = 0;
        }
        for (int cr = 0; cr <= 8; cr += 8)
            for (int cc = 0; cc <= 8; cc += 8) {
                int vr = cr == 0 ? 1 : 7, hc = cc == 0 ? 1 : 7; /* the corner's two neighbours */
                if (cell_at(g, cr, cc) == 3 - p && cell_at(g, vr, cc) == p && cell_at(g, cr, hc) == p &&
                    (to == vr * 9 + cc || to == cr * 9 + hc))
                    g->cell[cr * 9 + cc] = 0;
            }
    }
    g->ply += 1;
    if (!again) g->to_move = 3 - p;
    if (g->game == OR_WOLF && p == 2 && rt == 7) {
        finish(g, 2);
        return;
    }
    if (g->game == OR_HASAMI && hasami_line(g, p)) {
        finish(g, p);
        return;
    }
    if (move_legal(g, g->to_move, NULL) == 0) finish(g, p);
}

/* --------------------------------------------------------- legal actions --
 * legal[a] = 1 for each legal action a in [0, num_actions); returns the
 * count.  A finished game has no legal action.                           */
int oracle_legal(const ogame* g, uint8_t* legal) {
    int A = oracle_num_actions(g->game, g->rows, g->cols);
    int n = 0;
    memset(legal, 0, (size_t)A);
    if (g->outcome != OR_ONGOING) return 0;
    if (is_move_game(g->game)) return move_legal(g, g->to_move, legal);
    for (int i = 0; i < g->ncells; i++) {
        int ok = 0;
        if (g->cell[i] != 0) continue;
        switch (g->game) {
        case OR_TTT:
        case OR_HEX:
        case OR_GOMOKU:
        case OR_YAVALATH: ok = 1; break;
        case OR_PENTE: ok = g->ply > 0 || i == (g->rows / 2) * g->cols + g->cols / 2; break; /* first move: centre */
        case OR_LINE: {
            int r = i / g->cols, c = i % g->cols;
            ok = !(g->flags & OR_LINE_GRAVITY) || r == g->rows - 1 || at(g, r + 1, c) != 0;
            break;
        }
        case OR_C4: {
            int r = i / g->cols, c = i % g->cols;
            ok = (r == g->rows - 1) || (at(g, r + 1, c) != 0);
            break;
        }
        case OR_OTHELLO: ok = othello_cell_legal(g, g->to_move, i); break;
        }
        legal[i] = (uint8_t)ok;
        n += ok;
    }
    if (g->game == OR_OTHELLO && n == 0) {
        legal[g->ncells] = 1; /* force_pass */
        n = 1;
    }
    return n;
}

static void finish(ogame* g, int outcome) { g->outcome = outcome; }

/* Rewards for [P1, P2] from the final outcome (PGX shape). */
void oracle_rewards(const ogame* g, float* rew2) {
    rew2[0] = rew2[1] = 0.0f;
    if (g->outcome == OR_P1) { rew2[0] = 1.0f; rew2[1] = -1.0f; }
    if (g->outcome == OR_P2) { rew2[0] = -1.0f; rew2[1] = 1.0f; }
}

/* ----------------------------------------------------------------- step --
 * Apply one action for the player to move.  Returns 0 on success, 1 when the
 * game was already over (a no-op), -1 for an illegal action (the game ends
 * and the mover loses).                                                   */
int oracle_apply(ogame* g, int action) {
    uint8_t legal[OR_MAXACTIONS];
    int A, p;
    if (g->outcome != OR_ONGOING) return 1;
    A = oracle_num_actions(g->game, g->rows, g->cols);
    oracle_legal(g, legal);
    p = g->to_move;
    if (action < 0 || action >= A || !legal[action]) {
        g->illegal = 1;
        finish(g, 3 - p);
        return -1;
    }
    if (is_move_game(g->game)) {
        move_apply(g, action);
        if (g->outcome == OR_ONGOING && g->ply >= oracle_ply_cap(g->game, g->rows, g->cols)) finish(g, OR_CAPPED);
        return 0;
    }
    if (g->game == OR_OTHELLO && action == g->ncells) {
        g->passes += 1;
    } else {
        int r, c;
        cell_rc(g, action, &r, &c);
        g->cell[action] = (int8_t)p;
        if (g->game == OR_PENTE) {
            /* custodial capture of exactly two opponent stones: the new stone,
             * two opponent stones, then one of the mover's, along any of the
             * eight directions; the two are removed and counted */
            for (int d = 0; d < 8; d++) {
                int r1 = r + ODR[d], c1 = c + ODC[d], r2 = r + 2 * ODR[d], c2 = c + 2 * ODC[d];
                int r3 = r + 3 * ODR[d], c3 = c + 3 * ODC[d];
                if (in_board(g, r3, c3) && at(g, r1, c1) == 3 - p && at(g, r2, c2) == 3 - p && at(g, r3, c3) == p) {
                    g->cell[cell_id(g, r1, c1)] = 0;
                    g->cell[cell_id(g, r2, c2)] = 0;
                    g->captures[p] += 2;
                }
            }
        }
        if (g->game == OR_OTHELLO) {
            int runs[8];
            for (int d = 0; d < 8; d++) runs[d] = custodial_run(g, p, r, c, d);
            for (int d = 0; d < 8; d++)
                for (int k = 1; k <= runs[d]; k++) g->cell[(r + k * ODR[d]) * g->cols + c + k * ODC[d]] = (int8_t)p;
            g->passes = 0;
        }
    }
    g->ply += 1;
    g->to_move = 3 - p;
    /* end rules, in order: win first, then draw */
    switch (g->game) {
    case OR_TTT:
        if (has_line(g, p, 3)) finish(g, p);
        else if (board_full(g)) finish(g, OR_DRAW);
        break;
    case OR_C4:
        if (has_line(g, p, 4)) finish(g, p);
        else if (board_full(g)) finish(g, OR_DRAW);
        break;
    case OR_HEX:
        if (hex_connects(g, p)) finish(g, p);
        break;
    case OR_GOMOKU:
        if (has_line_exact(g, p, 5)) finish(g, p);
        else if (board_full(g)) finish(g, OR_DRAW);
        break;
    case OR_PENTE:
        if (has_line(g, p, 5) || g->captures[p] >= 10) finish(g, p);
        else if (board_full(g)) finish(g, OR_DRAW);
        break;
    case OR_LINE: {
        int made = (g->flags & OR_LINE_EXACT) ? has_line_exact(g, p, g->line) : has_line(g, p, g->line);
        if (made) finish(g, (g->flags & OR_LINE_MISERE) ? 3 - p : p);
        else if (board_full(g)) finish(g, OR_DRAW);
        break;
    }
    case OR_YAVALATH:
        if (has_line(g, p, 4)) finish(g, p);
        else if (has_line(g, p, 3)) finish(g, 3 - p);
        else if (board_full(g)) finish(g, OR_DRAW);
        break;
    case OR_OTHELLO:
        if (g->passes >= 2) {
            int n1 = 0, n2 = 0;
            for (int i = 0; i < g->ncells; i++) {
                n1 += g->cell[i] == 1;
                n2 += g->cell[i] == 2;
            }
            finish(g, n1 > n2 ? OR_P1 : (n2 > n1 ? OR_P2 : OR_DRAW));
        }
        break;
    }
    if (g->outcome == OR_ONGOING && g->ply >= oracle_ply_cap(g->game, g->rows, g->cols)) finish(g, OR_CAPPED);
    return 0;
}

/* -------------------------------------------------------------- playout --
 * Uniform-random playout of one env.  Each ply: collect the legal actions
 * in ascending id; if the only one is the forced pass, play it without a
 * draw; otherwise draw r = draw(seed, env, ply) and play the k-th legal
 * action with k = pick(r, count).  Stops at the end of the game or, when
 * stop_ply >= 0, once ply == stop_ply.                                    */
void oracle_playout(ogame* g, uint64_t seed, uint64_t env, int stop_ply) {
    uint8_t legal[OR_MAXACTIONS];
    int A = oracle_num_actions(g->game, g->rows, g->cols);
    while (g->outcome == OR_ONGOING && (stop_ply < 0 || g->ply < stop_ply)) {
        int n = oracle_legal(g, legal);
        int action = -1;
        if (g->game == OR_OTHELLO && legal[g->ncells]) {
            action = g->ncells;
        } else {
            uint32_t k = oracle_pick(oracle_draw(seed, env, (uint64_t)g->ply), (uint32_t)n);
            for (int a = 0; a < A; a++)
                if (legal[a]) {
                    if (k == 0) { action = a; break; }
                    k--;
                }
        }
        oracle_apply(g, action);
    }
}

/* -------------------------------------------------------- batch helpers --
 * State arrays used to move positions in and out of the oracle:
 *   board[e*ncells + i]  int8 cell values
 *   to_move[e] (1/2), ply[e], passes[e], outcome[e] (-1 ongoing)            */
/* Pente keeps its capture counts in the passes slot of the state arrays:
 * passes[e] = captures by P1 + 16 * (captures by P2) / 2 ... stored as
 * (captures by P1 / 2) | (captures by P2 / 2) << 4 (pairs, at most 15). */
static void load_state(ogame* g, int game, int rows, int cols, int64_t e, const int8_t* board, const int8_t* to_move,
                       const int16_t* ply, const int8_t* passes, const int8_t* outcome) {
    oracle_init(g, game, rows, cols);
    memcpy(g->cell, board + e * g->ncells, (size_t)g->ncells);
    g->to_move = to_move[e];
    g->ply = ply[e];
    g->outcome = outcome[e];
    if (game == OR_PENTE) {
        int v = (uint8_t)passes[e];
        g->captures[1] = 2 * (v & 15);
        g->captures[2] = 2 * (v >> 4);
    } else if (game == OR_DRAUGHTS) {
        g->pending = passes[e] - 1; /* the passes slot holds pending + 1 */
    } else {
        g->passes = passes[e];
    }
}

static void store_state(const ogame* g, int64_t e, int8_t* board, int8_t* to_move, int16_t* ply, int8_t* passes,
                        int8_t* outcome) {
    if (board) memcpy(board + e * g->ncells, g->cell, (size_t)g->ncells);
    if (to_move) to_move[e] = (int8_t)g->to_move;
    if (ply) ply[e] = (int16_t)g->ply;
    if (passes) {
        if (g->game == OR_PENTE) {
            int a = g->captures[1] / 2, b = g->captures[2] / 2;
            passes[e] = (int8_t)((a > 15 ? 15 : a) | ((b > 15 ? 15 : b) << 4));
        } else if (g->game == OR_DRAUGHTS) {
            passes[e] = (int8_t)(g->pending + 1);
        } else {
            passes[e] = (int8_t)g->passes;
        }
    }
    if (outcome) outcome[e] = (int8_t)g->outcome;
}

/* Playouts from the start position for envs env_offset .. env_offset+n-1.
 * Outputs (each nullable): final boards, outcome, final ply.               */
int oracle_rollout_start(int game, int rows, int cols, int64_t n, int64_t env_offset, uint64_t seed, int8_t* board,
                         int8_t* outcome, int16_t* plies) {
    ogame g;
    if (oracle_check_params(game, rows, cols) != 0) return -1;
    for (int64_t e = 0; e < n; e++) {
        oracle_init(&g, game, rows, cols);
        oracle_playout(&g, seed, (uint64_t)(env_offset + e), -1);
        store_state(&g, e, board, NULL, plies, NULL, outcome);
    }
    return 0;
}

/* Playouts (or partial playouts up to stop_ply[e] when stop_ply is given)
 * from the given states, which are updated in place.                      */
int oracle_rollout_from(int game, int rows, int cols, int64_t n, int64_t env_offset, uint64_t seed, int8_t* board,
                        int8_t* to_move, int16_t* ply, int8_t* passes, int8_t* outcome, const int16_t* stop_ply) {
    ogame g;
    if (oracle_check_params(game, rows, cols) != 0) return -1;
    for (int64_t e = 0; e < n; e++) {
        load_state(&g, game, rows, cols, e, board, to_move, ply, passes, outcome);
        oracle_playout(&g, seed, (uint64_t)(env_offset + e), stop_ply ? stop_ply[e] : -1);
        store_state(&g, e, board, to_move, ply, passes, outcome);
    }
    return 0;
}

/* One step for each env with the given actions; rewards [n][2] float,
 * terminated [n] (1 when the game is over after the step), error [n] (1 for
 * an illegal action).  States are updated in place.                        */
int oracle_step_batch(int game, int rows, int cols, int64_t n, int8_t* board, int8_t* to_move, int16_t* ply,
                      int8_t* passes, int8_t* outcome, const int32_t* actions, float* rewards, uint8_t* terminated,
                      uint8_t* error) {
    ogame g;
    if (oracle_check_params(game, rows, cols) != 0) return -1;
    for (int64_t e = 0; e < n; e++) {
        int st;
        load_state(&g, game, rows, cols, e, board, to_move, ply, passes, outcome);
        st = oracle_apply(&g, actions[e]);
        if (st == 1) {
            rewards[2 * e] = rewards[2 * e + 1] = 0.0f;
        } else if (g.outcome == OR_ONGOING || g.outcome == OR_CAPPED) {
            rewards[2 * e] = rewards[2 * e + 1] = 0.0f;
        } else {
            oracle_rewards(&g, rewards + 2 * e);
        }
        terminated[e] = (uint8_t)(g.outcome != OR_ONGOING);
        error[e] = (uint8_t)(st == -1);
        store_state(&g, e, board, to_move, ply, passes, outcome);
    }
    return 0;
}

/* Legal-action masks for a batch of states: legal[e*A + a]. */
int oracle_legal_batch(int game, int rows, int cols, int64_t n, const int8_t* board, const int8_t* to_move,
                       const int16_t* ply, const int8_t* passes, const int8_t* outcome, uint8_t* legal) {
    ogame g;
    int A = oracle_num_actions(game, rows, cols);
    if (oracle_check_params(game, rows, cols) != 0) return -1;
    for (int64_t e = 0; e < n; e++) {
        load_state(&g, game, rows, cols, e, board, to_move, ply, passes, outcome);
        oracle_legal(&g, legal + e * A);
    }
    return 0;
}

/* Start positions for a batch (board, to_move, ply, passes, outcome). */
int oracle_reset_batch(int game, int rows, int cols, int64_t n, int8_t* board, int8_t* to_move, int16_t* ply,
                       int8_t* passes, int8_t* outcome) {
    ogame g;
    if (oracle_init(&g, game, rows, cols) != 0) return -1;
    for (int64_t e = 0; e < n; e++) store_state(&g, e, board, to_move, ply, passes, outcome);
    return 0;
}

/* Mixed batch: desc[e] packs game | rows << 8 | cols << 16 for env e. */
int oracle_rollout_mixed(const int32_t* desc, int64_t n, int64_t env_offset, uint64_t seed, int8_t* outcome,
                         int16_t* plies) {
    ogame g;
    for (int64_t e = 0; e < n; e++) {
        int game = desc[e] & 0xFF, rows = (desc[e] >> 8) & 0xFF, cols = (desc[e] >> 16) & 0xFF;
        if (game == OR_LINE) game |= ((desc[e] >> 24) & 15) << 8 | ((desc[e] >> 28) & 7) << 12;
        if (oracle_init(&g, game, rows, cols) != 0) return -1;
        oracle_playout(&g, seed, (uint64_t)(env_offset + e), -1);
        outcome[e] = (int8_t)g.outcome;
        plies[e] = (int16_t)g.ply;
    }
    return 0;
}

/* ---------------------------------------------------------------- perft --
 * Number of action sequences of length depth from the start position in
 * which no position before the last action is finished.                    */
static uint64_t perft_rec(const ogame* g, int depth) {
    uint8_t legal[OR_MAXACTIONS];
    int A, n;
    uint64_t total = 0;
    if (depth == 0) return 1;
    if (g->outcome != OR_ONGOING) return 0;
    A = oracle_num_actions(g->game, g->rows, g->cols);
    n = oracle_legal(g, legal);
    (void)n;
    for (int a = 0; a < A; a++) {
        if (!legal[a]) continue;
        ogame child = *g;
        oracle_apply(&child, a);
        total += perft_rec(&child, depth - 1);
    }
    return total;
}

/* Perft by turns: an action after which the same player moves again (a
 * Draughts capture that must continue) does not use up a level, so a whole
 * multi-capture counts as one move, as published Draughts perft counts do. */
static uint64_t perft_turns_rec(const ogame* g, int depth) {
    uint8_t legal[OR_MAXACTIONS];
    int A;
    uint64_t total = 0;
    if (depth == 0) return 1;
    if (g->outcome != OR_ONGOING) return 0;
    A = oracle_num_actions(g->game, g->rows, g->cols);
    oracle_legal(g, legal);
    for (int a = 0; a < A; a++) {
        if (!legal[a]) continue;
        ogame child = *g;
        oracle_apply(&child, a);
        if (child.outcome == OR_ONGOING && child.to_move == g->to_move) total += perft_turns_rec(&child, depth);
        else total += perft_turns_rec(&child, depth - 1);
    }
    return total;
}

uint64_t oracle_perft_turns(int game, int rows, int cols, int depth) {
    ogame g;
    if (oracle_init(&g, game, rows, cols) != 0) return 0;
    return perft_turns_rec(&g, depth);
}

uint64_t oracle_perft(int game, int rows, int cols, int depth) {
    ogame g;
    if (oracle_init(&g, game, rows, cols) != 0) return 0;
    return perft_rec(&g, depth);
}

/* ------------------------------------------------- Tic-Tac-Toe enumeration --
 * Walks every complete game; counts[length*3 + outcome] with outcome
 * 0 draw, 1 X (P1) win, 2 O (P2) win, length in 0..9.                      */
static void ttt_walk(const ogame* g, uint64_t* counts) {
    uint8_t legal[16];
    if (g->outcome != OR_ONGOING) {
        counts[g->ply * 3 + g->outcome] += 1;
        return;
    }
    oracle_legal(g, legal);
    for (int a = 0; a < 9; a++) {
        if (!legal[a]) continue;
        ogame child = *g;
        oracle_apply(&child, a);
        ttt_walk(&child, counts);
    }
}

void oracle_ttt_enumerate(uint64_t* counts /* [10*3] */) {
    ogame g;
    memset(counts, 0, sizeof(uint64_t) * 30);
    oracle_init(&g, OR_TTT, 3, 3);
    ttt_walk(&g, counts);
}

/* ================================================================ MCTS ==
 * UCT (Kocsis and Szepesvari, ECML 2006): Monte-Carlo tree search with the
 * UCB1 rule in the tree and a uniform-random playout from each new leaf, the
 * agent of App. F's GAVEL-like evaluation ("MCTS with UCB1", a number of
 * iterations per move, each = traversal, expansion, random rollout).
 *
 * The paper leaves the details open; this is the definition both sides
 * implement:
 *   - a node holds N (visits) and W (reward in half points, for the player
 *     who made the move into the node: win 2, draw or capped 1, loss 0);
 *   - iteration i of a search with key K: key_i = sm(K ^ i); from the root,
 *     while the game is not over: if the node has untried legal actions, draw
 *     k = pick(sm(~key_i), count) and expand the k-th untried action in
 *     ascending action id (a forced pass is the only legal action), then stop
 *     descending; otherwise go to the child with the largest
 *     UCB1 = W / (2N) + T[N_parent] / sqrt(N), T[m] = c * sqrt(ln m),
 *     the smallest action id on a tie;
 *   - from the reached node, a uniform-random playout with draws
 *     sm(key_i ^ ply) (as the benchmark's playouts, with key_i as the env key);
 *   - every node on the path from the reached node up to, not including, the
 *     root gets N += 1 and its mover's reward; the root gets N += 1;
 *   - the move: the root child with the most visits, then the largest W, then
 *     the smallest action id.
 * A match plays such searches for both sides: match m (global index) has the
 * key K_m = sm(sm(seed) ^ m); the search at ply t has key sm(K_m ^ (t+1) << 32);
 * a position with a single legal action is played without a search.       */
typedef struct {
    int parent, action, mover, first_child, next_sibling;
    uint32_t N, W;
} onode;

static void playout_key(ogame* g, uint64_t key) {
    uint8_t legal[OR_MAXACTIONS];
    int A = oracle_num_actions(g->game, g->rows, g->cols);
    while (g->outcome == OR_ONGOING) {
        int n = oracle_legal(g, legal), action = -1;
        if (g->game == OR_OTHELLO && legal[g->ncells]) {
            action = g->ncells;
        } else {
            uint32_t k = oracle_pick(oracle_sm(key ^ (uint64_t)g->ply), (uint32_t)n);
            for (int a = 0; a < A; a++)
                if (legal[a]) {
                    if (k == 0) { action = a; break; }
                    k--;
                }
        }
        oracle_apply(g, action);
    }
}

static uint32_t reward_half_points(int outcome, int mover) {
    if (outcome == mover) return 2;
    if (outcome == OR_DRAW || outcome == OR_CAPPED) return 1;
    return 0;
}

/* One search from *root; returns the chosen action.  visits / wins, when
 * not NULL, receive the root children's N and W by action id. */
static int mcts_search(const ogame* root, uint64_t key, int iters, double c, uint32_t* visits, uint32_t* wins) {
    int A = oracle_num_actions(root->game, root->rows, root->cols);
    onode* nd = (onode*)calloc((size_t)iters + 1, sizeof(onode));
    uint8_t* tried = (uint8_t*)calloc(((size_t)iters + 1) * (size_t)A, 1);
    double* T = (double*)calloc((size_t)iters + 2, sizeof(double));
    uint8_t legal[OR_MAXACTIONS];
    int count = 1, best = -1;
    for (int m = 1; m <= iters + 1; m++) T[m] = c * sqrt(log((double)m));
    nd[0].parent = -1;
    nd[0].action = -1;
    nd[0].first_child = -1;
    nd[0].next_sibling = -1;
    for (int i = 0; i < iters; i++) {
        uint64_t ki = oracle_sm(key ^ (uint64_t)i);
        ogame g = *root;
        int x = 0;
        while (g.outcome == OR_ONGOING) {
            int untried = 0;
            oracle_legal(&g, legal);
            for (int a = 0; a < A; a++) untried += legal[a] && !tried[(size_t)x * A + a];
            if (untried > 0) {
                uint32_t k = oracle_pick(oracle_sm(~ki), (uint32_t)untried);
                int a = 0, y = count++;
                for (a = 0; a < A; a++)
                    if (legal[a] && !tried[(size_t)x * A + a]) {
                        if (k == 0) break;
                        k--;
                    }
                tried[(size_t)x * A + a] = 1;
                nd[y].parent = x;
                nd[y].action = a;
                nd[y].mover = g.to_move;
                nd[y].first_child = -1;
                nd[y].next_sibling = nd[x].first_child;
                nd[x].first_child = y;
                oracle_apply(&g, a);
                x = y;
                break;
            } else {
                int pick = -1;
                double bq = 0.0;
                for (int y = nd[x].first_child; y >= 0; y = nd[y].next_sibling) {
                    double q = (double)nd[y].W / (2.0 * (double)nd[y].N) + T[nd[x].N] / sqrt((double)nd[y].N);
                    if (pick < 0 || q > bq || (q == bq && nd[y].action < nd[pick].action)) {
                        pick = y;
                        bq = q;
                    }
                }
                oracle_apply(&g, nd[pick].action);
                x = pick;
            }
        }
        playout_key(&g, ki);
        for (int y = x; y > 0; y = nd[y].parent) {
            nd[y].N += 1;
            nd[y].W += reward_half_points(g.outcome, nd[y].mover);
        }
        nd[0].N += 1;
    }
    for (int y = nd[0].first_child; y >= 0; y = nd[y].next_sibling) {
        if (visits) visits[nd[y].action] = nd[y].N;
        if (wins) wins[nd[y].action] = nd[y].W;
        if (best < 0 || nd[y].N > nd[best].N || (nd[y].N == nd[best].N && nd[y].W > nd[best].W) ||
            (nd[y].N == nd[best].N && nd[y].W == nd[best].W && nd[y].action < nd[best].action))
            best = y;
    }
    {
        int action = best >= 0 ? nd[best].action : -1;
        free(nd);
        free(tried);
        free(T);
        return action;
    }
}

static uint64_t search_key(uint64_t seed, int64_t match, int ply) {
    uint64_t km = oracle_sm(oracle_sm(seed) ^ (uint64_t)match);
    return km ^ ((uint64_t)(ply + 1) << 32);
}

/* One search per state of the batch (states in the batch-helper layout);
 * action[e] = chosen action (-1 when the game is over); visits / wins
 * [e*A + a] = N / W of the root child for action a (0 if not expanded). */
int oracle_mcts_search(int game, int rows, int cols, int64_t n, int64_t env_offset, uint64_t seed, int iters, double c,
                       const int8_t* board, const int8_t* to_move, const int16_t* ply, const int8_t* passes,
                       const int8_t* outcome, int32_t* action, uint32_t* visits, uint32_t* wins) {
    int A;
    if (oracle_check_params(game, rows, cols) != 0 || iters < 1) return -1;
    A = oracle_num_actions(game, rows, cols);
    for (int64_t e = 0; e < n; e++) {
        ogame g;
        load_state(&g, game, rows, cols, e, board, to_move, ply, passes, outcome);
        if (visits) memset(visits + e * A, 0, (size_t)A * sizeof(uint32_t));
        if (wins) memset(wins + e * A, 0, (size_t)A * sizeof(uint32_t));
        action[e] = g.outcome != OR_ONGOING
                        ? -1
                        : mcts_search(&g, oracle_sm(search_key(seed, env_offset + e, g.ply)), iters, c,
                                      visits ? visits + e * A : NULL, wins ? wins + e * A : NULL);
    }
    return 0;
}

/* Matches between two agents (iters_p1 for P1's moves, iters_p2 for P2's)
 * from the start position.  Per match: the outcome, the plies, the turns with
 * more than one legal action, and the cells occupied at some point. */
int oracle_mcts_play(int game, int rows, int cols, int64_t n, int64_t env_offset, uint64_t seed, int iters_p1,
                     int iters_p2, double c, int8_t* outcome, int16_t* plies, int16_t* agency, int16_t* coverage) {
    uint8_t legal[OR_MAXACTIONS];
    if (oracle_check_params(game, rows, cols) != 0 || iters_p1 < 1 || iters_p2 < 1) return -1;
    for (int64_t e = 0; e < n; e++) {
        ogame g;
        uint8_t ever[OR_MAXCELLS];
        int turns = 0, covered = 0, A;
        oracle_init(&g, game, rows, cols);
        A = oracle_num_actions(g.game, rows, cols);
        for (int i = 0; i < g.ncells; i++) ever[i] = g.cell[i] != 0;
        while (g.outcome == OR_ONGOING) {
            int k = oracle_legal(&g, legal), a = -1;
            if (k > 1) {
                turns++;
                a = mcts_search(&g, oracle_sm(search_key(seed, env_offset + e, g.ply)),
                                g.to_move == 1 ? iters_p1 : iters_p2, c, NULL, NULL);
            } else {
                for (int j = 0; j < A; j++)
                    if (legal[j]) a = j;
            }
            oracle_apply(&g, a);
            for (int i = 0; i < g.ncells; i++) ever[i] |= g.cell[i] != 0;
        }
        for (int i = 0; i < g.ncells; i++) covered += ever[i];
        outcome[e] = (int8_t)g.outcome;
        plies[e] = (int16_t)g.ply;
        agency[e] = (int16_t)turns;
        coverage[e] = (int16_t)covered;
    }
    return 0;
}
