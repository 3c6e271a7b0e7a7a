// ludax_internal.cuh -- host-side definitions shared by the library's
// translation units (the env handle and the game dispatcher).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/ludax.h"
#include "ludax_state.cuh"

struct ludax_env {
    int32_t game, rows, cols, cells, num_actions, mask_words, planes;
    int64_t n, env_offset;
    cudaStream_t stream;
    int device, num_sms;
    uint64_t* d_planes;
    uint32_t* d_meta;
    unsigned long long* d_counters;  // [0] refill cursor, [1] illegal, [2] capped, [3] spare
    int32_t desc;                    // game descriptor (with the line game's parameters)
    void* d_tree;                    // MCTS node slabs (grown on demand)
    size_t tree_bytes;
    double* d_ucb;                   // UCB1 table T[m] = c * sqrt(ln m)
    int ucb_len;
    double ucb_c;
    uint8_t* d_stage;                // device staging of ludax_rollout_host (grown on demand)
    size_t stage_bytes;
};

namespace ludax {

template <class G>
struct Tag {
    using type = G;
};

// Calls f(Tag<G>{}) for the game type of (game, n); LUDAX_ERR_* if unknown.
template <class F>
int dispatch_game(int game, int rows, int cols, F&& f) {
    switch (game) {
    case LUDAX_GAME_TTT: return (rows == 3 && cols == 3) ? f(Tag<TTT>{}) : LUDAX_ERR_SIZE;
    case LUDAX_GAME_C4: return (rows == 6 && cols == 7) ? f(Tag<C4>{}) : LUDAX_ERR_SIZE;
    case LUDAX_GAME_OTHELLO: return (rows == 8 && cols == 8) ? f(Tag<Othello>{}) : LUDAX_ERR_SIZE;
    case LUDAX_GAME_HEX:
        if (rows != cols) return LUDAX_ERR_SIZE;
        switch (rows) {
        case 2: return f(Tag<Hex<2>>{});
        case 3: return f(Tag<Hex<3>>{});
        case 4: return f(Tag<Hex<4>>{});
        case 5: return f(Tag<Hex<5>>{});
        case 6: return f(Tag<Hex<6>>{});
        case 7: return f(Tag<Hex<7>>{});
        case 8: return f(Tag<Hex<8>>{});
        case 9: return f(Tag<Hex<9>>{});
        case 10: return f(Tag<Hex<10>>{});
        case 11: return f(Tag<Hex<11>>{});
        default: return LUDAX_ERR_SIZE;
        }
    case LUDAX_GAME_GOMOKU: return (rows == 15 && cols == 15) ? f(Tag<Gomoku>{}) : LUDAX_ERR_SIZE;
    case LUDAX_GAME_PENTE: return (rows == 19 && cols == 19) ? f(Tag<Pente>{}) : LUDAX_ERR_SIZE;
    case LUDAX_GAME_YAVALATH: return (rows == 9 && cols == 9) ? f(Tag<Yavalath>{}) : LUDAX_ERR_SIZE;
    case LUDAX_GAME_LINE:
        return (rows >= 1 && cols >= 1 && rows * (cols + 1) <= 128) ? f(Tag<LineGame>{}) : LUDAX_ERR_SIZE;
    case LUDAX_GAME_WOLF_SHEEP: return (rows == 8 && cols == 8) ? f(Tag<WolfSheep>{}) : LUDAX_ERR_SIZE;
    case LUDAX_GAME_DRAUGHTS: return (rows == 8 && cols == 8) ? f(Tag<Draughts>{}) : LUDAX_ERR_SIZE;
    case LUDAX_GAME_HASAMI_SHOGI: return (rows == 9 && cols == 9) ? f(Tag<HasamiShogi>{}) : LUDAX_ERR_SIZE;
    default: return LUDAX_ERR_GAME;
    }
}

// Per-env descriptors (game | rows << 8 | cols << 16 | line << 24 | flags << 28)
// grouped by kernel instance ("buckets"): 0 TTT, 1 C4, 2 Othello, 3 + k Hex
// (k + 2) x (k + 2), 13 Gomoku, 14 Pente, 15 Yavalath, 16 the parametric line
// game (any parameters), 17 Wolf and Sheep, 18 Draughts, 19 Dai Hasami Shogi.
// Returns the bucket, -1 for an unknown game or -2 for a board size the
// game's kernel does not take.
constexpr int kDescBuckets = 20;
__host__ __device__ inline int desc_bucket(int32_t d) {
    if (d < 0) return -1;
    const int game = d & 0xFF, rows = (d >> 8) & 0xFF, cols = (d >> 16) & 0xFF;
    if (game == LUDAX_GAME_LINE) {
        const int L = (d >> 24) & 15, mx = rows > cols ? rows : cols;
        return (rows >= 1 && cols >= 1 && rows * (cols + 1) <= 128 && L >= 2 && L <= mx) ? 16 : -2;
    }
    if ((d >> 24) != 0) return -1;
    switch (game) {
    case LUDAX_GAME_TTT: return (rows == 3 && cols == 3) ? 0 : -2;
    case LUDAX_GAME_C4: return (rows == 6 && cols == 7) ? 1 : -2;
    case LUDAX_GAME_OTHELLO: return (rows == 8 && cols == 8) ? 2 : -2;
    case LUDAX_GAME_HEX: return (rows == cols && rows >= 2 && rows <= 11) ? 3 + rows - 2 : -2;
    case LUDAX_GAME_GOMOKU: return (rows == 15 && cols == 15) ? 13 : -2;
    case LUDAX_GAME_PENTE: return (rows == 19 && cols == 19) ? 14 : -2;
    case LUDAX_GAME_YAVALATH: return (rows == 9 && cols == 9) ? 15 : -2;
    case LUDAX_GAME_WOLF_SHEEP: return (rows == 8 && cols == 8) ? 17 : -2;
    case LUDAX_GAME_DRAUGHTS: return (rows == 8 && cols == 8) ? 18 : -2;
    case LUDAX_GAME_HASAMI_SHOGI: return (rows == 9 && cols == 9) ? 19 : -2;
    default: return -1;
    }
}

// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per (kernel, device); LUDAX_OK or LUDAX_ERR_CUDA.
int ensure_smem_limit(const void* kernel, size_t bytes);
// SMs of the current device (0 on error).
int device_sms();

// dense BF16 layer on tcgen05 tensor cores (ludax_umma.cu):
// out = bf16(relu(A . B^T + bias)), A [M][K], B [N][K] row-major
bool umma_dense_supported(int M, int N, int K);
int umma_dense_relu(const void* A, const void* B, const float* bias, void* out, int M, int N, int K, int ldo,
                    cudaStream_t s);
// The same layer with row pitches lda / ldb (K may be a prefix of the rows:
// columns past K are not read) and, with w3 non-null (N BF16 weights), the
// head fused into the epilogue: zpart[m * (N / 256) + j] = sum over the j-th
// 256 columns of bf16(relu(.))[m][n] * w3[n]; the rows are stored as well
// when out is non-null (at least one of out and w3 must be given).
int umma_dense_relu_ex(const void* A, int lda, const void* B, int ldb, const float* bias, void* out, int ldo,
                       const void* w3, float* zpart, int M, int N, int K, cudaStream_t s);
// Both hidden layers (512 wide) and the head in one launch for inference:
// zpart[m * 4 + j] = sum over columns 128 j .. 128 j + 127 of
// bf16(relu(bf16(relu(X W1^T + b1)) W2^T + b2))[m][n] * w3[n].  X [M][ldx]
// (first K1 columns read), W1 [512][ldw1], W2 [512][512]; scratch holds
// umma_mlp_scratch_rows() rows of 512 BF16 (layer 1's rows pass through it).
int umma_mlp_scratch_rows();
int umma_mlp_head(const void* X, int ldx, int K1, const void* W1, int ldw1, const float* b1, const void* W2,
                  const float* b2, const void* w3, float* zpart, void* scratch, int scratch_rows, int M,
                  cudaStream_t s);
// The same launch for training: layer 1's rows kept in H1 [M][512] and layer
// 2's in H2 [M][512] (BF16), zpart as above (four partials per row), and
// (h1bits non-null) which of H1's values are non-zero as M * 16 words in the
// layout h1bits_index below.
int umma_mlp_train(const void* X, int ldx, int K1, const void* W1, int ldw1, const float* b1, const void* W2,
                   const float* b2, const void* w3, float* zpart, void* H1, void* H2, uint32_t* h1bits, int M,
                   cudaStream_t s);
// Index of the word of a bit mask over an [M][N] matrix (N a multiple of
// 32) that holds row r, column j, as bit j % 32.  A 32-row group keeps its
// rows' words for columns 32 w .. 32 w + 31 side by side (row r % 32 at
// offset r % 32), so the 32 rows of a group read or write one column word as
// 128 consecutive bytes.
__host__ __device__ __forceinline__ long long h1bits_index(int r, int j, int N) {
    return ((long long)(r >> 5) * (N >> 5) + (j >> 5)) * 32 + (r & 31);
}

// The value net's backward contractions on tcgen05 (ludax_umma.cu).
// umma_grad_mask: out[m][n] = bf16(mask[m][n] > 0 ? sum_k A[m][k] B[k][n] : 0)
// with A [M][K], B [K][N], mask and out [M][N], all row-major BF16.  With
// colpart non-null it also leaves the column sums of out (the stored BF16
// values, summed in FP32) as umma_grad_colrows(M, N) partial rows of N
// floats: every row of out is counted in exactly one of them, and each
// partial row is written in full.
int umma_grad_mask(const void* A, const void* B, const void* mask, void* out, int M, int N, int K, float* colpart,
                   cudaStream_t s);
// The same with the mask given as bits (h1bits_index layout, bit set where
// the value is non-zero): the mask then costs M * N / 8 bytes of reads
// instead of M * N * 2.
int umma_grad_maskbits(const void* A, const void* B, const uint32_t* maskbits, void* out, int M, int N, int K,
                       float* colpart, cudaStream_t s);
int umma_grad_colrows(int M, int N);  // 0 on error; at most 4 * SMs
// umma_grad_weights: part[p][m][n] = FP32 sum over the p-th of *splits_out
// contiguous K ranges of A[k][m] B[k][n]; A [K][lda], B [K][ldb] row-major
// BF16; part holds part_floats floats (the split count is capped by it).
// last_use: bit 0 / bit 1 -- A / B is read for the last time in the
// training step (its lines are the first L2 gives up).  umma_grad_mask and
// umma_grad_maskbits always treat A (dZ2) that way.
int umma_grad_weights(const void* A, int lda, const void* B, int ldb, int M, int N, int K, float* part,
                      long long part_floats, int* splits_out, cudaStream_t s, int last_use);

// Programmatic dependent launch.  A kernel started with launch_dependent is
// scheduled as the CTAs of the kernel before it on the stream exit (each
// exit counts as that CTA's trigger), so its CTAs fill the SMs the previous
// kernel's tail leaves idle, and run up to their pdl_wait(), which returns
// once that kernel (and so everything before it) has completed and its
// memory is visible: it must come before the kernel's first global load or
// store.  For an ordinary launch it is a no-op.  (Triggering at the start of
// a kernel instead let the next kernel's waiting CTAs take SM resources
// early and made the training step slower.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

template <class... KArgs, class... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                             Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// An NVTX range over one C-ABI call, named after it, so that a profiler or
// tracer attributes the call's host work and launches to it; with no tool
// attached a push or pop is one check of a function pointer.
struct ApiRange {
    explicit ApiRange(const char* name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
    ApiRange(const ApiRange&) = delete;
    ApiRange& operator=(const ApiRange&) = delete;
};

}  // namespace ludax
