/*
 * ludax.h -- C-ABI of the B300 batched board-game engine.
 *
 * The engine runs the hot path of Ludax's compiled board-game environments
 * (Ludax, arXiv 2506.22609): batched game stepping over very many parallel
 * environments and uniform-random playouts to termination, for Tic-Tac-Toe,
 * Connect Four, Reversi/Othello and Hex (rules: App. C of the paper).  The
 * interface mirrors the paper's environment API (a PGX-shaped env with
 * init/step, a fixed-size legal-action mask, rewards and a terminated flag;
 * Sec. 1, Sec. 3.4 and Sec. 4) with every call batched over num_envs envs.
 *
 * Conventions shared by every entry point:
 *   - Status: each function returns LUDAX_OK (0) or a negative LUDAX_ERR_*.
 *     Nothing throws or aborts across the ABI.  Arguments are validated on
 *     the host before any launch; a rejected call launches nothing.
 *   - Ownership: every pointer named *_dev is device memory owned by the
 *     caller (for instance a torch tensor's data_ptr()), valid until the
 *     launched work has finished.  The env owns its own state buffer, which
 *     it allocates in ludax_env_create and frees in ludax_env_destroy.
 *   - Asynchrony: launches are asynchronous on the env's CUDA stream (the
 *     cudaStream_t passed as void*; NULL = the legacy default stream).  Use
 *     ludax_sync, or the caller's own stream synchronisation, before reading
 *     outputs on the host.
 *   - Cells: the canonical cell id of row r, column c is r*cols + c with row
 *     0 at the TOP of the board (the numbering of the paper's English
 *     Draughts listing, App. A, where P1 moves up from cells 40..62).
 *   - Actions: one action per cell, the destination cell (Sec. 3.4; for
 *     Connect Four the legal cells are the empty cells on the bottom row or
 *     directly above an occupied cell).  Reversi adds one pass action with
 *     id rows*cols (= 64), legal only when no cell is (force_pass, App. B).
 *   - Players: P1 moves first; cell values 0 empty, 1 P1, 2 P2.
 *   - Outcome codes: LUDAX_OUTCOME_*.  Rewards are float32 pairs [P1, P2]:
 *     (+1,-1) P1 wins, (-1,+1) P2 wins, (0,0) draw or not finished.
 *   - Randomness: the uniform-random policy draws r = sm(key ^ ply) with
 *     key = sm(sm(seed) ^ env), sm the splitmix64 output function (Steele,
 *     Lea and Flood 2014), env the GLOBAL env index (env_offset + local
 *     index) and ply the env's ply counter (passes included).  The move is
 *     the k-th legal cell in ascending cell id with k = ((r >> 32) * n) >> 32
 *     for n legal cells.  A forced pass consumes a ply but no draw.  Every
 *     trajectory is therefore reproducible from (seed, env, start state),
 *     independent of launch shape, thread mapping or refill order.
 */
#ifndef LUDAX_H
#define LUDAX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status -- */
#define LUDAX_OK 0
#define LUDAX_ERR_ARG (-1)     /* null pointer, bad count, bad flag       */
#define LUDAX_ERR_GAME (-2)    /* unknown game id or descriptor            */
#define LUDAX_ERR_SIZE (-3)    /* board size not supported for the game    */
#define LUDAX_ERR_CUDA (-4)    /* a CUDA runtime call failed               */
#define LUDAX_ERR_TIMEOUT (-5) /* ludax_sync deadline passed              */
#define LUDAX_ERR_ALIGN (-6)   /* a device pointer is misaligned           */
#define LUDAX_ERR_NOMEM (-7)   /* device allocation failed                 */

/* ------------------------------------------------------------- games -- */
#define LUDAX_GAME_TTT 0     /* Tic-Tac-Toe 3x3, line of 3                 */
#define LUDAX_GAME_C4 1      /* Connect Four 6x7, gravity, line of 4       */
#define LUDAX_GAME_OTHELLO 2 /* Reversi/Othello 8x8, flips, forced pass    */
#define LUDAX_GAME_HEX 3     /* Hex n x n rhombus, 2 <= n <= 11            */
#define LUDAX_GAME_GOMOKU 4  /* Gomoku 15x15, a line of exactly five wins  */
#define LUDAX_GAME_PENTE 5   /* Pente 19x19, five in a row or ten captured
                                stones win; P1's first move is the centre  */
#define LUDAX_GAME_YAVALATH 6 /* Yavalath, 61-cell hexagon (board params
                                 9x9): four in a row wins, three loses     */
#define LUDAX_GAME_LINE 7     /* parametric line game on any rows x cols board
                                 with rows*(cols+1) <= 128: place on an empty
                                 cell (with gravity if LUDAX_LINE_GRAVITY); a
                                 line of at least `line` stones (exactly, with
                                 LUDAX_LINE_EXACT) wins -- loses, with
                                 LUDAX_LINE_MISERE; a full board draws    */
#define LUDAX_LINE_EXACT 1
#define LUDAX_LINE_GRAVITY 2
#define LUDAX_LINE_MISERE 4
/* Games whose pieces move (App. C): an action is from * cells + to, so
 * num_actions = cells^2; P1 starts at the bottom; the mover wins when the
 * player to move next has no legal action; capped (OUTCOME_CAPPED) after 200
 * plies (Sec. 6 stops unbounded games after 200 turns).                   */
#define LUDAX_GAME_WOLF_SHEEP 8    /* 8x8: four sheep (P1, cells 56/58/60/62) step
                                      diagonally up, the wolf (P2, cell 3) steps
                                      diagonally either way; the wolf wins on
                                      the bottom row                          */
#define LUDAX_GAME_DRAUGHTS 9      /* English Draughts 8x8: men on the dark cells
                                      of rows 5-7 (P1) and 0-2 (P2); forced
                                      hops, multi-hops as extra turns of the
                                      same piece, crowning on the far row     */
#define LUDAX_GAME_HASAMI_SHOGI 10 /* Dai Hasami Shogi 9x9: rook slides or hops
                                      over an adjacent piece; custodial and
                                      corner captures; five in a row outside
                                      the mover's two home rows wins          */

/* ---------------------------------------------------------- outcomes -- */
#define LUDAX_OUTCOME_ONGOING (-1)
#define LUDAX_OUTCOME_DRAW 0
#define LUDAX_OUTCOME_P1 1
#define LUDAX_OUTCOME_P2 2
#define LUDAX_OUTCOME_CAPPED 3 /* ply cap hit: 9/42/128/n*n never for a correct engine; Pente
                                  2,000 and the move games 200 (games of unbounded length) */

/* ------------------------------------------------------ rollout flags -- */
#define LUDAX_ROLLOUT_FROM_START 1u /* play from the start position; stored state not read */
#define LUDAX_ROLLOUT_WRITE_BACK 2u /* store each env's final state back into the env       */

typedef struct {
    int32_t rows;
    int32_t cols;
    int32_t line;  /* LUDAX_GAME_LINE: line length, 2..min(15, max(rows, cols)); else 0 */
    int32_t flags; /* LUDAX_GAME_LINE: LUDAX_LINE_* bits; else 0                   */
} ludax_board_params;

typedef struct ludax_env ludax_env;

/* A batch of positions in canonical form, all arrays on the device:
 *   board   int8  [num_envs][cells]      cell values 0/1/2 (cells = rows*cols;
 *                                        Yavalath: the 61 cells of the hexagon,
 *                                        row by row, left to right); Draughts
 *                                        kings are 3 (P1) and 4 (P2)
 *   to_move int8  [num_envs]             1 or 2
 *   ply     int16 [num_envs]             plies played (passes included)
 *   passes  int8  [num_envs]             consecutive passes (Reversi); Pente:
 *                                        captured pairs, P1's in the low 4 bits,
 *                                        P2's in the high 4 bits; Draughts: 1 +
 *                                        the cell of the piece that must hop
 *                                        again (0 if none); else 0
 *   outcome int8  [num_envs]             LUDAX_OUTCOME_*                      */
typedef struct {
    int8_t* board;
    int8_t* to_move;
    int16_t* ply;
    int8_t* passes;
    int8_t* outcome;
} ludax_state_view;

/* Launch shape of the persistent playout kernels (see ludax_autotune). */
typedef struct {
    int32_t block_threads;   /* threads per block: 32..512, multiple of 32           */
    int32_t blocks_per_sm;   /* resident blocks per SM for the persistent grid, >= 1;
                                0 = one thread per env (no persistence)               */
    int32_t envs_per_thread; /* envs each thread advances together (ILP): 1 or 2
                                (mixed batches: 2 only with blocks_per_sm 0)         */
    int32_t hex_nbr_table;   /* Hex neighbour test: 0 = bit shifts, 1 = shared-memory
                                table of per-cell neighbour masks                     */
    int32_t compact_every;   /* single-game playouts only (0 for mixed batches): 0 =
                                off; else every `compact_every` plies each block packs
                                its unfinished envs into its lowest warps through shared
                                memory (idle warps stop issuing) and refills the freed
                                slots from the queue; needs envs_per_thread 1         */
    int32_t threads_per_env; /* lanes cooperating on one env: 0 or 1 = one lane per env
                                (every game and path); 2 or 4 = Hex single-game
                                ludax_rollout only (the board's four 32-bit words split
                                across the lanes, draws and end tests shared by warp
                                shuffles; same results bit for bit); needs
                                envs_per_thread 1 and compact_every 0                 */
    int32_t lanes_per_warp;  /* lanes of each warp that hold envs: 0 or 32 = all; 8 or
                                16 = ludax_rollout and mixed batches with
                                blocks_per_sm 0, the rest of the warp idle (small,
                                latency-bound batches: fewer envs share a warp's issue
                                slots and divergent branches); needs compact_every 0
                                and one lane per env; envs per warp = lanes_per_warp x
                                envs_per_thread                                        */
} ludax_launch_cfg;

/* ---------------------------------------------------------------------------
 * Environment lifetime.
 *
 * ludax_env_create: a batch of num_envs independent envs of one game, in the
 * start position (Sec. 3.1: empty board, Reversi's four discs at D4/E5 white =
 * P2 on cells 27/36 and D5/E4 black = P1 on cells 35/28; P1 to move).
 *   game       LUDAX_GAME_*
 *   p          board size: TTT 3x3, C4 6x7, Othello 8x8, Hex n x n (2..11),
 *              Gomoku 15x15, Pente 19x19, Yavalath 9x9 (the hexagon's axial grid),
 *              Wolf and Sheep 8x8, Draughts 8x8, Dai Hasami Shogi 9x9
 *   num_envs   1 .. 2^31-1
 *   env_offset global index of env 0 (keys the random draws; lets several
 *              GPUs or calls cover disjoint env ranges), >= 0
 *   stream     cudaStream_t for every launch of this env (NULL = default)
 * Allocates the env's state on the current device.  Returns LUDAX_ERR_GAME,
 * LUDAX_ERR_SIZE, LUDAX_ERR_ARG or LUDAX_ERR_NOMEM without side effects.   */
int ludax_env_create(ludax_env** out, int32_t game, const ludax_board_params* p, int64_t num_envs, int64_t env_offset,
                     void* stream);
/* Frees the env's state (synchronises its stream first).  NULL is a no-op. */
int ludax_env_destroy(ludax_env* env);
/* Rebind the env to another stream (same device). */
int ludax_env_set_stream(ludax_env* env, void* stream);

/* Sizes of the env's action space: num_actions = cells (+1 pass for
 * Reversi; cells^2 for the move games); mask_words = ceil(cells / 64) words
 * per env in legal masks (ceil(cells^2 / 64) for the move games).          */
int ludax_env_sizes(const ludax_env* env, int32_t* num_actions, int32_t* mask_words, int64_t* num_envs);

/* ---------------------------------------------------------------------------
 * ludax_reset: put envs back in the start position.  env_mask_dev (uint8
 * [num_envs], nullable) selects the envs to reset; NULL resets all.        */
int ludax_reset(ludax_env* env, const uint8_t* env_mask_dev);

/* ludax_legal_mask: the legal-action mask of each env (Sec. 3.2: the legal
 * action mask function of the play mechanic; Sec. 4: fixed size).
 *   mask_dev       uint64 [num_envs][mask_words]: bit (i % 64) of word i/64
 *                  set when cell i is a legal destination; all zero for a
 *                  finished env
 *   pass_legal_dev uint8 [num_envs], nullable: 1 when the pass action is the
 *                  (only) legal action (Reversi with no legal cell)          */
int ludax_legal_mask(ludax_env* env, uint64_t* mask_dev, uint8_t* pass_legal_dev);

/* ludax_step: apply actions_dev[e] (int32 action ids) to every env, then
 * apply the effects (Reversi flips), the end rules in order (win before
 * draw, Sec. 3.3) and write
 *   rewards_dev    float32 [num_envs][2] rewards [P1, P2] of this step
 *   terminated_dev uint8 [num_envs] 1 when the env is finished after it.
 * A finished env is left unchanged with zero rewards.  An illegal action
 * (out of range, occupied, not supported by gravity, not custodial, or a pass
 * while a cell is legal) ends the env: the mover gets -1, the opponent +1,
 * the outcome names the opponent, and the env's illegal-action counter (see
 * ludax_counters) is incremented.  The paper does not define this case; the
 * rule follows the PGX environments Ludax builds on.                       */
int ludax_step(ludax_env* env, const int32_t* actions_dev, float* rewards_dev, uint8_t* terminated_dev);

/* ludax_random_step: one step of the uniform-random policy for every env
 * (the random-policy benchmark of Sec. 6), drawing each action as described
 * at the top of this file with the given seed.  Outputs as ludax_step.
 * Repeated calls reproduce ludax_rollout's trajectories ply for ply.       */
int ludax_random_step(ludax_env* env, uint64_t seed, float* rewards_dev, uint8_t* terminated_dev);

/* ludax_rollout: uniform-random playout of every env to the end of its game
 * in one fused persistent kernel (state stays in registers; lanes take a new
 * env when theirs finishes).
 *   seed           keys the draws
 *   flags          LUDAX_ROLLOUT_FROM_START | LUDAX_ROLLOUT_WRITE_BACK
 *   stop_ply_dev   int16 [num_envs], nullable: stop an env as soon as its
 *                  ply counter reaches stop_ply (outcome then -1)
 *   outcome_dev    int8 [num_envs], nullable: LUDAX_OUTCOME_* at the end
 *   plies_dev      int16 [num_envs], nullable: the env's final ply counter
 *                  (game length, passes included, when played from start)
 *   cfg            launch shape, nullable = the built-in default           */
int ludax_rollout(ludax_env* env, uint64_t seed, uint32_t flags, const int16_t* stop_ply_dev, int8_t* outcome_dev,
                  int16_t* plies_dev, const ludax_launch_cfg* cfg);

/* ludax_rollout_host: ludax_rollout for positions held on the host -- the
 * whole round trip in one call.  Enqueues on the env's stream, in order: the
 * copy of the packed state (planes_host uint64 [words_per_env][num_envs],
 * meta_host uint32 [num_envs]; the layout of ludax_get_state_bits) to device
 * staging owned by the env, loading it as ludax_set_state_bits does, the
 * playout of every env to its end (seed, launch shape cfg, nullable), and the
 * copies of outcome_host int8 [num_envs] and plies_host int16 [num_envs] back;
 * returns without waiting (ludax_sync, or the stream, tells when the outputs
 * are in place).  Host buffers should be page-locked for the copies to run
 * asynchronously.  The playout kernel loads the packed positions itself; the
 * env's stored state is not changed.  The staging (num_envs x (8 x
 * words_per_env + 8) bytes at most) is allocated on the first call and kept
 * until ludax_env_destroy; growing it synchronises the stream. */
int ludax_rollout_host(ludax_env* env, const uint64_t* planes_host, const uint32_t* meta_host, uint64_t seed,
                       int8_t* outcome_host, int16_t* plies_host, const ludax_launch_cfg* cfg);
/* The same with one host buffer each way (one copy each way):
 *   in_host  planes (8 x words_per_env x num_envs bytes, the layout above)
 *            followed by meta (4 x num_envs bytes)
 *   out_host outcome (num_envs bytes), one pad byte when num_envs is odd,
 *            then plies (2 x num_envs bytes)
 * Both 8-byte aligned, page-locked for asynchronous copies. */
int ludax_rollout_host_packed(ludax_env* env, const void* in_host, void* out_host, uint64_t seed,
                              const ludax_launch_cfg* cfg);

/* ludax_rollout_value: for every env, R independent uniform-random playouts
 * from its current state; playout j (0 <= j < R) draws with seed + j.
 *   value_dev float32 [num_envs]: mean result from P1's view (win 1, draw
 *             0.5, loss 0) -- the Monte-Carlo value estimate of the position.
 * The env's state is not modified.                                         */
int ludax_rollout_value(ludax_env* env, uint64_t seed, int32_t R, float* value_dev, const ludax_launch_cfg* cfg);

/* ludax_get_state / ludax_set_state: copy every env's position out of / into
 * the canonical view (all five arrays required, device memory).  set_state
 * validates nothing about reachability; it rebuilds the engine's internal
 * form (bitboards, Hex edge-connected sets) from the cell values.          */
int ludax_get_state(ludax_env* env, const ludax_state_view* dst);
int ludax_set_state(ludax_env* env, const ludax_state_view* src);

/* Packed form of the same canonical state, for moving many positions at
 * two bits per cell instead of a byte (a library interface; the paper's
 * environments hold the board as arrays):
 *   planes_dev uint64 [words_per_env][num_envs] (plane-major across envs):
 *              V planes, one per nonzero cell value v = 1 .. V (V = 4 for
 *              Draughts -- men 1/2, kings 3/4 -- else 2), each W =
 *              ceil(cells / 64) words in canonical cell order: bit c % 64 of
 *              word (v - 1) * W + c / 64 is set iff cell c holds v
 *   meta_dev   uint32 [num_envs]: ply (bits 0-15) | (to_move - 1) << 16 |
 *              the state view's passes byte << 17 | (outcome + 1) << 25
 * words_per_env = V * W (ludax_state_bits_words).  set_state_bits ignores
 * bits past the last cell and, like set_state, validates nothing about
 * reachability; both are asynchronous on the env's stream.  LUDAX_ERR_ARG
 * on null pointers, LUDAX_ERR_ALIGN unless planes are 8- and meta 4-byte
 * aligned. */
int ludax_state_bits_words(const ludax_env* env, int32_t* words_per_env);
int ludax_get_state_bits(ludax_env* env, uint64_t* planes_dev, uint32_t* meta_dev);
int ludax_set_state_bits(ludax_env* env, const uint64_t* planes_dev, const uint32_t* meta_dev);

/* ludax_counters: host-visible totals since creation (synchronises the
 * env's stream): illegal actions seen by ludax_step, envs that hit the ply
 * cap.  Either pointer may be NULL.                                         */
int ludax_counters(ludax_env* env, int64_t* illegal_actions, int64_t* capped);

/* ludax_sync: wait for the env's stream with a deadline by polling
 * (cudaStreamQuery); LUDAX_ERR_TIMEOUT when timeout_ms passes first
 * (the work is not cancelled).  timeout_ms < 0 waits without a deadline.  */
int ludax_sync(ludax_env* env, int64_t timeout_ms);

const char* ludax_status_string(int status);

/* ---------------------------------------------------------------------------
 * Mixed-game batches: one persistent launch over envs of different games and
 * board sizes, each env's game given by an int32 descriptor
 *   desc = game | rows << 8 | cols << 16   (LUDAX_DESC(g, r, c))
 *   desc = LUDAX_GAME_LINE | rows << 8 | cols << 16 | line << 24 | flags << 28
 *          (LUDAX_DESC_LINE(r, c, line, flags))
 * for any game and board size ludax_env_create accepts.  Results match
 * per-game ludax_rollout calls from the start position with the same (seed,
 * global env index) bit for bit.                                           */
#define LUDAX_DESC(g, r, c) ((int32_t)((g) | ((r) << 8) | ((c) << 16)))
/* descriptor of the parametric line game: line length in bits 24-27, flags in 28-30 */
#define LUDAX_DESC_LINE(r, c, line, flags) \
    ((int32_t)(LUDAX_GAME_LINE | ((r) << 8) | ((c) << 16) | ((line) << 24) | ((flags) << 28)))

typedef struct ludax_mixed_plan ludax_mixed_plan;

/* Build a plan for desc_dev (int32 [num_envs], device; read during this call
 * and by later launches, so keep it alive and unchanged): validates every
 * descriptor (LUDAX_ERR_GAME / LUDAX_ERR_SIZE name the first bad one through
 * bad_index, nullable), groups env ids by game into a work queue so that a
 * warp runs one game at a time, and captures the launch (queue counter reset
 * + persistent kernel) into a CUDA graph on `stream`.
 *   cfg     launch shape, nullable = built-in default (or a ludax_autotune
 *           result)                                                         */
int ludax_mixed_plan_create(ludax_mixed_plan** out, const int32_t* desc_dev, int64_t num_envs, int64_t env_offset,
                            const ludax_launch_cfg* cfg, void* stream, int64_t* bad_index);
/* Replay the captured graph with a new seed and output buffers:
 * outcome_dev int8 [num_envs], plies_dev int16 [num_envs].                */
int ludax_mixed_plan_launch(ludax_mixed_plan* plan, uint64_t seed, int8_t* outcome_dev, int16_t* plies_dev);
/* The plan's playout with the batch in HOST memory (the end-to-end form of
 * the mixed-batch benchmark of Sec. 6): desc_host int32 [num_envs] (any
 * descriptors, not only those the plan was built from) is copied to the
 * device, the game-grouped work queue is rebuilt there (no host round trip),
 * the envs are played with the plan's launch shape and env_offset, and
 * outcome_host int8 [num_envs] and plies_host int16 [num_envs] are copied
 * back -- all asynchronously on the plan's stream, so the host buffers must
 * stay valid until the stream reaches this call (pinned memory lets the
 * copies overlap other streams' work).  The plan's first host-buffer call
 * allocates its device staging (11 bytes per env + 1 KiB) and one pinned
 * word.  An env whose descriptor is invalid is not played (outcome -1,
 * plies 0); ludax_mixed_plan_sync reports it.  Calls on one plan are ordered
 * by its stream; the replayed graph (ludax_mixed_plan_launch) keeps its own
 * queue and is unaffected.                                                 */
int ludax_mixed_plan_launch_host(ludax_mixed_plan* plan, uint64_t seed, const int32_t* desc_host,
                                 int8_t* outcome_host, int16_t* plies_host);
/* Wait for the plan's stream; if the last host-buffer launch met an invalid
 * descriptor, return LUDAX_ERR_GAME or LUDAX_ERR_SIZE for the first one and
 * its index through bad_index (nullable; -1 when none).                    */
int ludax_mixed_plan_sync(ludax_mixed_plan* plan, int64_t* bad_index);
int ludax_mixed_plan_destroy(ludax_mixed_plan* plan);

/* Same work without a graph: one direct launch (used to validate the graph). */
int ludax_rollout_mixed(const int32_t* desc_dev, int64_t num_envs, int64_t env_offset, uint64_t seed,
                        int8_t* outcome_dev, int16_t* plies_dev, const ludax_launch_cfg* cfg, void* stream);

/* Allocation-free variant of ludax_rollout_mixed, for callers that cannot
 * allocate device memory: plugins running inside a host framework whose
 * memory pool already owns the device's memory (a cudaMalloc of ours could
 * fail or fragment that pool), and serving loops where cudaFree would
 * synchronise the whole device and stall every other stream.  (The paper has
 * no counterpart: this is a deployment entry point of this library.)
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *     Its scratch -- the game-grouped work queue and the claim cursors -- is a
 *     static device array of 4 MiB plus 1 KiB, held by every GPU that
 *     loads this library until the process exits.
 *   - num_envs at most 1,048,576 (2^20): larger batches return LUDAX_ERR_SIZE
 *     before anything is launched.
 *   - The first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress (which may load the library's device code) and
 *     keeps it for the process; make that first call before any stream
 *     capture on the device.  The kept address is not refreshed, so do not
 *     use this entry point on a device after cudaDeviceReset.
 *   - Every call shares the one array: the call resets the counters it needs
 *     and overwrites the queue, so calls whose work overlaps on the GPU (other
 *     streams or threads) race and must be serialised by the caller.
 *   - Blocks until the descriptors are validated: it synchronises `stream`
 *     after a small device-to-host read of the bucket counts (and one more
 *     read of the bad descriptor when there is one); the playout itself
 *     stays asynchronous on `stream`.
 * Arguments, results and errors as ludax_rollout_mixed; bad_index (nullable)
 * receives the index of the first invalid descriptor, else -1.            */
int ludax_rollout_mixed_noalloc(const int32_t* desc_dev, int64_t num_envs, int64_t env_offset, uint64_t seed,
                                int8_t* outcome_dev, int16_t* plies_dev, const ludax_launch_cfg* cfg, void* stream,
                                int64_t* bad_index);

/* Autotuner: times every candidate launch shape (block_threads x
 * blocks_per_sm x hex_nbr_table, and for one thread per env envs_per_thread
 * x lanes_per_warp; ludax_autotune_candidates lists them) on the given mixed batch
 * with CUDA events (warm-up, then the median of `reps` launches) and returns
 * the fastest in best_out; best_ms_out (nullable) its median time.
 * ms_table_out (nullable, host) receives each candidate's median in
 * candidate order; n_candidates_out (nullable) their number.               */
int ludax_autotune(const int32_t* desc_dev, int64_t num_envs, uint64_t seed, int32_t reps, void* stream,
                   ludax_launch_cfg* best_out, float* best_ms_out, float* ms_table_out, int32_t* n_candidates_out);
/* The candidate list ludax_autotune walks (host memory, count returned). */
int ludax_autotune_candidates(ludax_launch_cfg* out, int32_t max_out);

/* Autotuner for ludax_rollout on one env batch (from the start position, no
 * write-back; the env's stored state is not touched): walks block_threads x
 * blocks_per_sm x envs_per_thread x compact_every, and for Hex also
 * hex_nbr_table and threads_per_env 2 and 4 (the candidates of
 * ludax_autotune_env_candidates, in that order), timing each like
 * ludax_autotune.  ms_table_out (nullable) needs room for 512 floats.      */
int ludax_autotune_env(ludax_env* env, uint64_t seed, int32_t reps, ludax_launch_cfg* best_out, float* best_ms_out,
                       float* ms_table_out, int32_t* n_candidates_out);
/* The candidate list ludax_autotune_env walks for this env's game (host
 * memory, at most max_out written, the full count returned).              */
int ludax_autotune_env_candidates(const ludax_env* env, ludax_launch_cfg* out, int32_t max_out);

/* ---------------------------------------------------------------------------
 * Value network that truncates playouts (the learned part built on the
 * engine; the paper's own agents, Sec. 7, are AlphaZero ResNets, which this
 * library does not provide).
 *
 * Input row of a position: bf16 1.0 at column c for each P1 stone on cell c,
 * at column cells + c for each P2 stone, at column 2*cells when P1 is to
 * move; zero up to in_pad = round_up(2*cells + 1, 128) columns.  Layers:
 * in_pad -> 512 ReLU -> 512 ReLU -> 1, v = tanh(z), predicted probability that
 * P1 wins p = (v + 1) / 2.  BF16 weights and activations, FP32 accumulation;
 * FP32 master weights and Adam (beta1 0.9, beta2 0.999, eps 1e-8).  Loss:
 * mean over the batch of (p - y)^2.
 *
 * Parameters are one flat FP32 vector in the order
 *   W1 [512][in_pad], b1 [512], W2 [512][512], b2 [512], w3 [512], b3 [1].
 * Batches B must be multiples of 128 and at most max_batch.  All pointers are
 * device memory; the net works on its own stream.                           */
typedef struct ludax_net ludax_net;

int ludax_net_create(ludax_net** out, int32_t cells, int64_t max_batch, void* stream);
int ludax_net_destroy(ludax_net* net);
int ludax_net_sizes(const ludax_net* net, int32_t* in_pad, int32_t* hidden, int64_t* num_params);
/* set_params copies params_dev (float [num_params]) and resets Adam's moments
 * and step count; get_params copies the FP32 masters out. */
int ludax_net_set_params(ludax_net* net, const float* params_dev);
int ludax_net_get_params(ludax_net* net, float* params_dev);
/* The whole training state, for checkpoints: the FP32 parameters, Adam's
 * first and second moments (each float [num_params], device memory, owned by
 * the caller) and the number of Adam steps taken (host).  get copies them out
 * on the net's stream (any pointer may be null to skip it); set restores all
 * of them (none null; 0 <= steps < 2^31) and the BF16 weight copies, so that
 * the next train step is the one that followed get.  LUDAX_ERR_ARG on a bad
 * argument, LUDAX_ERR_CUDA if a copy fails. */
int ludax_net_get_state(ludax_net* net, float* params_dev, float* m_dev, float* v_dev, int64_t* steps);
int ludax_net_set_state(ludax_net* net, const float* params_dev, const float* m_dev, const float* v_dev,
                        int64_t steps);
/* Which kernels run the hidden-layer contractions:
 *   1 (default) tcgen05/TMEM: a forward runs both layers and the head in one
 *     launch, layer 1's rows passing through L2 to layer 2 (without labels,
 *     ludax_net_forward and ludax_truncated_value, through a scratch; in
 *     training into H1, kept with layer 2's rows for the backward pass); the
 *     backward pass's three contractions (dZ1 = (dZ2 W2) * [H1 > 0] and the
 *     weight gradients over the batch, split into FP32 partial sums) run on
 *     tcgen05 too, and one launch reduces the partials and applies Adam; an
 *     input width that is not a multiple of 256 keeps dW1 on the mma.sync
 *     kernel;
 *   2 tcgen05/TMEM, always as two layer launches (the head fused into the
 *     second one's epilogue): the form used for inference when the scratch
 *     cannot be allocated, selectable for comparison; the backward pass as
 *     in 1;
 *   0 the mma.sync kernel for every contraction (kept for comparison).
 * Results agree to FP32 rounding order across the three. */
int ludax_net_set_tensor_path(ludax_net* net, int32_t use_tcgen05);
/* p_dev float [B]: predicted P(P1 wins) for the input rows x_dev (bf16 bits,
 * uint16 [B][in_pad], 16-byte aligned). */
int ludax_net_forward(ludax_net* net, const uint16_t* x_dev, int64_t B, float* p_dev);
/* Gradient of the loss against labels y_dev (float [B]) into grad_dev (float
 * [num_params], nullable) and the loss into loss_dev (float [1], nullable);
 * the parameters are not changed. */
int ludax_net_grad(ludax_net* net, const uint16_t* x_dev, const float* y_dev, int64_t B, float* grad_dev,
                   float* loss_dev);
/* One Adam step with learning rate lr on the batch; loss_dev as above. */
int ludax_net_train_step(ludax_net* net, const uint16_t* x_dev, const float* y_dev, int64_t B, float lr,
                         float* loss_dev);
/* The net input row of every env's current position into x_dev (uint16
 * [num_envs][ld], ld >= 2*cells+1, ld % 8 == 0, 16-byte aligned). */
int ludax_pack_inputs(ludax_env* env, uint16_t* x_dev, int32_t ld);
/* Truncated value estimate of every env's current position: K continuations
 * of up to `plies` uniform-random plies (continuation j draws as playout j of
 * ludax_rollout_value with this seed); a continuation that ends the game
 * counts its result (win 1, draw 0.5, loss 0 for P1), otherwise the net's p
 * at the leaf.  value_dev float [num_envs] = mean over the K continuations.
 * The env and the net must share a stream and the env's board size. */
int ludax_truncated_value(ludax_env* env, ludax_net* net, uint64_t seed, int32_t K, int32_t plies, float* value_dev);

/* ------------------------------------------------------------- MCTS --
 * UCT agents (Kocsis and Szepesvari 2006): Monte-Carlo tree search with the
 * UCB1 rule and one uniform-random playout per iteration, and whole matches
 * between two such agents -- the agents of the GAVEL-like evaluation of
 * App. F (which fixes "MCTS with UCB1" and iterations = traversal,
 * expansion, random rollout; the rest is defined here):
 *   - a node holds N (visits) and W (reward in half points for the player
 *     who moved into it: win 2, draw or capped game 1, loss 0);
 *   - iteration i of a search with key K uses key_i = sm(K ^ i); from the
 *     root, while the game is not over: a node with untried legal actions
 *     expands the k-th of them in ascending action id, k = umulhi(top32(
 *     sm(~key_i)), count), and the descent stops; otherwise the descent
 *     follows the child with the largest W/(2N) + T[N_parent]/sqrt(N),
 *     T[m] = c * sqrt(ln m) (double, correctly rounded), the smallest action
 *     on a tie; a forced pass is the only action of its node;
 *   - a uniform-random playout from the reached node draws sm(key_i ^ ply)
 *     per ply (as ludax_rollout with key_i as the env key);
 *   - the reached node and its ancestors below the root get N += 1 and their
 *     mover's reward; the root gets N += 1;
 *   - the move played: the root child with the most visits, then the
 *     largest W, then the smallest action id.
 * The search of env / match m (global index, env_offset included) at ply t
 * has K = sm(sm(sm(seed) ^ m) ^ ((t + 1) << 32)), sm = splitmix64.  The
 * tree lives in a scratch buffer the env owns (grown on demand: num_envs *
 * (iterations + 1) * (16 + 8 * mask words) bytes; LUDAX_ERR_NOMEM if it
 * cannot be allocated).  One warp runs one search or one match; while the
 * root has untried actions the warp's lanes play up to 32 iterations at
 * once, with the result of the sequential definition above. */
#define LUDAX_MCTS_MAX_ITERS 4096

/* Allocates the env's tree scratch for searches of up to `iterations` and
 * uploads the UCB1 table for c (synchronising), so that later
 * ludax_mcts_search / ludax_mcts_play calls with at most that many
 * iterations and the same c allocate nothing and stay asynchronous. */
int ludax_mcts_reserve(ludax_env* env, int32_t iterations, double c);

/* One search per env from its current state (the env is not modified).
 *   iterations  1 .. LUDAX_MCTS_MAX_ITERS;  c >= 0 (UCB1's exploration
 *               constant; sqrt(2) is the textbook value)
 *   action_dev  int32 [num_envs]: the chosen action id (-1 if the game is
 *               over; the pass id for a forced pass)
 *   visits_dev, wins_dev  uint32 [num_envs][num_actions], nullable: N and W
 *               of the root's children by action id (0 for no child)      */
int ludax_mcts_search(ludax_env* env, uint64_t seed, int32_t iterations, double c, int32_t* action_dev,
                      uint32_t* visits_dev, uint32_t* wins_dev);

/* One match per env between two UCT agents: P1 searches with iters_p1
 * iterations per move, P2 with iters_p2; a position with a single legal
 * action is played without a search.  flags: LUDAX_ROLLOUT_FROM_START
 * (start position; otherwise the env's current state) | LUDAX_ROLLOUT_
 * WRITE_BACK (store the final positions).  Per env, each output nullable:
 *   outcome_dev   int8  LUDAX_OUTCOME_* at the end (CAPPED: not completed)
 *   plies_dev     int16 final ply counter
 *   agency_dev    int16 turns that had more than one legal action
 *   coverage_dev  int16 cells that held a piece at some point of the match */
int ludax_mcts_play(ludax_env* env, uint64_t seed, uint32_t flags, int32_t iters_p1, int32_t iters_p2, double c,
                    int8_t* outcome_dev, int16_t* plies_dev, int16_t* agency_dev, int16_t* coverage_dev);

/* Matches of any mix of games in one launch (one warp per match): env e
 * plays the game of desc_host[e] (LUDAX_DESC / LUDAX_DESC_LINE) from its
 * start position, P1 searching with iters_host[2e] iterations per move and
 * P2 with iters_host[2e + 1]; match e has the global index env_offset + e
 * (its keys as in ludax_mcts_play).  desc_host and iters_host are HOST
 * arrays, validated (the first bad index goes to bad_index, nullable) and
 * copied before the call returns; the outputs are device arrays [n] as in
 * ludax_mcts_play.  Scratch is allocated and freed in stream order on
 * `stream`; the call returns once the launch is enqueued. */
int ludax_mcts_play_mixed(const int32_t* desc_host, const int32_t* iters_host, int64_t n, int64_t env_offset,
                          uint64_t seed, double c, int8_t* outcome_dev, int16_t* plies_dev, int16_t* agency_dev,
                          int16_t* coverage_dev, void* stream, int64_t* bad_index);

/* Dense BF16 layer on the tcgen05 tensor cores (the value net's forward
 * layers): out[m][n] = bf16(relu(sum_k a[m][k] * b[n][k] + bias[n])), FP32
 * accumulation.  a uint16 (bf16 bits) [M][K], b [N][K], bias float [N], out
 * [M][ld_out]; M % 128 == 0, N % 256 == 0, K % 64 == 0, 16-byte aligned
 * pointers, ld_out % 8 == 0 (LUDAX_ERR_SIZE otherwise).  Asynchronous on
 * `stream`.  The kernel bounds every internal wait; an expired wait is
 * reported by ludax_device_error. */
int ludax_dense_bf16_relu(const uint16_t* a_dev, const uint16_t* b_dev, const float* bias_dev, uint16_t* out_dev,
                          int32_t M, int32_t N, int32_t K, int32_t ld_out, void* stream);
/* Reads and clears the device error word of the tensor-core kernels
 * (synchronising): LUDAX_OK, or LUDAX_ERR_TIMEOUT when a kernel gave up on
 * an internal wait since the last call; error_out (nullable) gets the word. */
int ludax_device_error(int32_t* error_out);
/* Self-test of that failure path, without a fault: launches one thread that
 * waits on an mbarrier nothing arrives at, gives up after limit_cycles
 * (1 .. 2e9 clock cycles) and sets bit 2 of the device error word, as a
 * tensor-core kernel does when an internal wait expires.  The next
 * ludax_device_error then returns LUDAX_ERR_TIMEOUT, and the context stays
 * usable.  Asynchronous on `stream`. */
int ludax_selftest_wait(int64_t limit_cycles, void* stream);

/* Integer-issue microbenchmark behind the playouts' roofline: one launch
 * over every SM at full occupancy in which each thread issues `iters` x 8
 * independent 32-bit ops of one kind -- 0 LOP3 (3-input logic), 1 IADD
 * (add.u32), 2 SHF (funnel shift), 3 IMAD (mad.lo.u32), 4 IMAD.HI
 * (mul.hi.u32), 5 LOP3 and IMAD on alternate chains -- as inline PTX.
 * ops_out (host, nullable) gets the number of thread-level ops; time the
 * launch on `stream` (asynchronous).  kind in 0 .. 5 and iters in
 * 1 .. 2^30; LUDAX_ERR_ARG otherwise. */
int ludax_int_peak(int32_t kind, int64_t iters, int64_t* ops_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LUDAX_H */
