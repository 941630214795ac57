// Internal definitions shared by the host code and the kernel files of libletkf.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/letkf.h"

namespace letkf {

// Bits of the device status word (latched until letkf_sync reads them).
enum : int {
    ST_NONFINITE = 1,   // a frame's slopes held a NaN or Inf; the frame was rejected
    ST_NOCONV = 2,      // an eigensolve hit its sweep limit
    ST_TIMEOUT = 4,     // a bounded wait on an mbarrier gave up
};

// Device-side domain tables, flattened over domains.  All indices are int32.
struct DomainTables {
    int n_dom = 0;
    int* own_off = nullptr;     // [n_dom+1] into own
    int* own = nullptr;         // owned valid-actuator indices
    int* obs_off = nullptr;     // [n_dom+1] into obs_sub / obs_corner (observed subapertures)
    int* obs_sub = nullptr;     // valid-subaperture index of each observed subaperture
    int* obs_corner = nullptr;  // 4 halo-local corner indices packed in bytes: (r,c) (r,c+1) (r+1,c) (r+1,c+1)
    int* halo_off = nullptr;    // [n_dom+1] into halo
    int* halo = nullptr;        // valid-actuator indices of the corners of the observed subapertures
    int* order = nullptr;       // [n_dom] processing order, most expensive first
};

struct GlobalState;   // global.cu: buffers and graph of the global path

// Host copy of the geometry and domains.
struct HostModel {
    int n_sub = 0;
    std::vector<uint8_t> sub_valid, act_valid;
    std::vector<int> sub_index, act_index;   // grid -> valid index or -1
    std::vector<int> sub_rc, act_rc;         // valid index -> (r, c)
    int n_act = 0, n_subv = 0;
    std::vector<int> own_off, own, obs_off, obs_sub, obs_corner, halo_off, halo, order;
    std::vector<int> block;                  // block index I * blocks_per_side + J of each domain
    int blocks_per_side = 0;
    int n_loc_max = 0, p_loc_max = 0, n_h_max = 0;
};

}  // namespace letkf

struct letkf_ctx {
    // parameters
    int n_sub = 0, m = 0, m_pad = 0, dom_sub = 0, halo = 0;
    int precision = 0, path = 0, obs_block = 1, device = 0;
    double a = 0, a2 = 0, sigma = 0, q_white = 0;
    unsigned long long seed = 0;
    cudaStream_t stream = nullptr;
    int sms = 0;
    // geometry
    letkf::HostModel host;
    int n_act = 0, n_subv = 0, n = 0, p = 0, n_dom = 0;
    letkf::DomainTables tab;
    // ensemble: X[cur] is the current state, X[cur ^ 1] the next one (rows of m_pad elements)
    void* X[2] = {nullptr, nullptr};
    int cur = 0;
    int phase = 0;                  // 0: forecast phase, 1: analysis phase
    unsigned long long frame = 0;
    // process noise
    void* Lq = nullptr;             // FP64 / FP32: device L, n_act x n_act row-major
    void* Xi = nullptr;             // normals: n_act x m_pad (FP64 / FP32) or 64-row BF16 tiles (mixed)
    // mixed precision: L as BF16 128 x 64 operand tiles (lower-triangle tiles only when L is lower
    // triangular) and the work items of the noise kernel
    void* Lt = nullptr;
    int* noise_items = nullptr;     // int4 per item: row block, first tile, end tile, partial slot
    int* noise_tabs = nullptr;      // per row block: first tile, items, first slot; split blocks
    void* noise_part = nullptr;     // partial sums of row blocks split over several items
    int noise_nb = 0, noise_np = 0, noise_tile_b = 0, noise_n_items = 0, noise_grid = 0, noise_n_rb = 0;
    void* V = nullptr;              // perturbations, n_act x m_pad (state type)
    // scratch of the plain path
    void* S = nullptr;              // observed anomalies / sigma, sum(p_loc) x m_pad
    void* dt = nullptr;             // innovations / sigma, sum(p_loc)
    void* G = nullptr;              // n_dom x m x m_pad Gram matrices
    void* b = nullptr;              // n_dom x m_pad
    void* W = nullptr;              // n_dom x m x m_pad transforms w_bar 1^T + T
    int* so_off = nullptr;          // [n_dom] slope row offset of each domain in S
    int total_slopes = 0;
    // device flags
    int* d_status = nullptr;        // latched status bits
    int* d_frame_bad = nullptr;     // current frame rejected
    int* d_queue = nullptr;         // fused kernel: [0] work queue, [1] CTAs done, [2] non-finite slope seen
    size_t device_bytes = 0;
    int fused_smem = 0;             // dynamic shared memory of the fused kernel
    int fused_grid = 0;
    int dual = 0;                   // fused analysis in observation space (m >= 128)
    void* scratch = nullptr;        // dual form: per-CTA halo anomalies, SMs x scratch_stride floats
    int scratch_stride = 0;
    // fused path: process noise of the next frame drawn on a side stream while the current
    // frame's kernel runs (double-buffered; v_frame[b] = frame whose draw buffer b holds)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_v_ready[2] = {nullptr, nullptr};
    cudaEvent_t ev_v_used[2] = {nullptr, nullptr};
    void* Vbuf[2] = {nullptr, nullptr};
    void* Xi_side = nullptr;
    unsigned long long v_frame[2] = {~0ull, ~0ull};
    // fused step as a CUDA graph (one per frame parity): the fused kernel and, on a forked branch,
    // the next frame's noise draw; captured for the ensemble buffer in use (gcur)
    int graph_on = 0;
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaGraphNode_t gnode_fused[2] = {nullptr, nullptr};
    cudaGraphNode_t gnode_normals[2] = {nullptr, nullptr};
    int gcur[2] = {-1, -1};
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaStream_t cap_stream = nullptr;      // capture only
    // global path (one domain, tiled tensor-core products)
    letkf::GlobalState* gstate = nullptr;
    int lq_lower = 0;               // the process-noise factor is lower triangular
    // differential-piston removal: per-domain entries of the boundary subapertures, the
    // least-squares operator K (n_dom x n_dom), per-domain residual sums and the raw prediction
    int piston = 0;
    int simt_q_max = 0;             // requested SIMT threshold (letkf_params.simt_q_max)
    int simt_q = 0, simt_ws = 0;    // fused path: the threshold in use and its workspace bytes
    void* pst_ent = nullptr;
    int* pst_off = nullptr;
    int pst_n_ent = 0;
    void* pst_K = nullptr;
    void* pst_g = nullptr;
    void* xhat = nullptr;
    // fused path, test instrument: the analysis of domain cap_dom writes its mean weights and
    // transform (or the transform's factors) to cap_dev (letkf_set_capture)
    float* cap_dev = nullptr;
    int cap_dom = -1;
    // fused path: this context's prediction when it is the second filter of letkf_step_pair
    void* pair_pred = nullptr;
    // FP32 / FP64 dense process noise: work items and tiles (int4), per-tile counters and partial
    // tiles of the split-K draw V = L xi
    void* rg_items = nullptr;
    void* rg_tiles = nullptr;
    int* rg_count = nullptr;
    void* rg_part = nullptr;
    int rg_n_items = 0;
    // stage timing
    int prof_on = 0;
    std::vector<int> prof_stage;            // stage of each record
    std::vector<cudaEvent_t> prof_ev;       // two events per record
    size_t prof_used = 0;
};

namespace letkf {

int state_bytes(const letkf_ctx* c);

enum Stage { STAGE_CHECK = 0, STAGE_NOISE = 1, STAGE_OBS = 2, STAGE_GRAM = 3, STAGE_EIG = 4,
             STAGE_TRANSFORM = 5, STAGE_FORECAST = 6, STAGE_FUSED = 7, STAGE_PISTON = 8 };
// Record the start / end of a stage on the context's stream (no-ops unless profiling).
void prof_begin(letkf_ctx* c, int stage);
void prof_end(letkf_ctx* c);

// plain.cu
int plain_analyze(letkf_ctx* c, const void* y, double sigma);
int plain_limits_ok(int precision, int m);
size_t plain_smem_bytes(const letkf_ctx* c, int which);

// misc.cu
int launch_precheck(letkf_ctx* c, const void* y);
int launch_forecast(letkf_ctx* c, const void* v_user, void* xpred, int in_analysis);
int draw_perturbations(letkf_ctx* c, unsigned long long frame);
// Normals of `frame` into xi, then V = L xi into v_out, on `stream`.
int draw_perturbations_on(letkf_ctx* c, unsigned long long frame, void* xi, void* v_out, cudaStream_t stream);
int init_ensemble(letkf_ctx* c, const double* L_host, const double* P0_host);
// Split-K work plan of the per-frame draw V = L xi (n x n factor, m members): items and tiles
// (4 ints each, filled when not null), partial-tile slots; rg_bytes: its device bytes.
struct RowGemmPlan {
    int n_items = 0, n_tiles = 0, n_slots = 0;
    size_t part_elems = 0;
};
RowGemmPlan rg_plan(int n, int m, bool lower, int* items, int* tiles);
size_t rg_bytes(int n, int m, bool lower, size_t eb);
// Node parameters of the normals kernel draw_perturbations_on launches (arguments held in *nn).
struct NormalsNode {
    cudaKernelNodeParams params;
    void* args[7];
    void* out;
    int ld, n_act, m;
    unsigned long long seed;
    uint32_t stream_id, frame;
};
int normals_node_params(letkf_ctx* c, unsigned long long frame, void* xi, NormalsNode* nn);

// global.cu: the global (single-domain) ETKF at large ensemble sizes
size_t global_bytes(int n_act, int n_subv, int m, bool dense, int sms);
int global_prepare(letkf_ctx* c);
void global_free(letkf_ctx* c);
int global_analyze(letkf_ctx* c, const void* y, double sigma);
int global_forecast(letkf_ctx* c, const void* v_user, void* xpred, int in_analysis);

// gemm.cu: tiled tensor-core GEMM, C = A B^T with tiled BF16 operands (128 x 64 tiles)
enum GemmEpilogue { GEMM_EPI_F32 = 0, GEMM_EPI_TILES = 1, GEMM_EPI_ADD_ROW = 2 };
struct GemmArgs {
    const uint8_t* a_hi;
    const uint8_t* a_lo;        // null: single BF16
    const uint8_t* b_hi;
    const uint8_t* b_lo;
    int a_nkb, b_nkb;           // column tiles per row tile of A and B
    int nkb;                    // K / 64 steps to run
    int split;                  // 1: hi hi + hi lo + lo hi
    int a_lower;                // 1: A is lower triangular (K steps past the row tile skipped)
    const int2* tiles;          // non-null: blockIdx.x takes output tile (row tile, column tile) tiles[x]
    int ksplit;                 // > 1: blockIdx.z takes one of ksplit contiguous shares of the K steps,
    size_t c_split_stride;      //   F32 output of share z at c + z * c_split_stride
    int b_mn;                   // 1: B is the second factor M itself (tiles of M, rows = K), read
                                //    MN-major: C = A M (BN = 64 only); 0: C = A B^T
    int M, N;                   // valid rows / columns of C
    int mode;                   // GemmEpilogue
    float* c;                   // F32 / ADD_ROW: C[row * ldc + col]
    int ldc;
    float alpha;
    uint8_t* o_hi;              // TILES: alpha C + beta I as a tiled operand with o_nkb column tiles
    uint8_t* o_lo;
    int o_nkb;
    float beta;
    unsigned int* dev;          // TILES: max |C - I| over valid entries (float bits, atomicMax)
    const float* add;           // ADD_ROW: per-row term
    const int* run;             // non-null: the launch does nothing when *run == 0
    int* next_flag;             // non-null: CTA (0,0) sets *next_flag = run && (*dev_in >= run_tol),
    unsigned int* dev_in;       //   and, when running, resets *dev_in, sets *z_final = z_index
    float run_tol;              //   and counts one step in *steps
    int* z_final;
    int z_index;
    int* steps;
    int* status;
};
size_t tiled_bytes(int rows, int cols);
int gemm_prepare();
int gemm_launch(const GemmArgs& g, int bn, int m_tiles, int n_tiles, cudaStream_t stream);
int to_tiles(const float* src, int R, int K, int ld, void* hi, void* lo, cudaStream_t stream);

// piston.cu: differential pistons between domains
size_t piston_bytes(const HostModel& h, int n_dom, int elem_bytes);
// The least-squares operator K (n_dom x n_dom, FP64, row-major), on the host.
int piston_operator_host(const HostModel& h, int n_dom, std::vector<double>* K);
int piston_prepare(letkf_ctx* c);
// After a frame whose prediction is in c->xhat: x_out = x_hat + P delta (x_out may be null) and,
// in the in-loop mode, the shift of the new state X (both instants).
int piston_launch(letkf_ctx* c, const void* y, void* xout, void* X, cudaStream_t stream);

// noise.cu: the mixed-precision draw V = L Xi on the tensor cores
struct NoisePlan {
    bool lower = false;
    int nb = 0, nk = 0, np = 0, n_tiles = 0, n_items = 0, n_slots = 0;
    size_t tile_b = 0, bytes = 0;    // bytes: device memory of the tiles, tables and partial sums
    std::vector<int> prefix, jn, jslot, items;
};
bool lower_triangular(const double* L, int n);
NoisePlan noise_plan(int n_act, int m, bool lower);
size_t noise_xi_bytes(int n_act, int m);
int noise_prepare(letkf_ctx* c, const double* L_host);
int noise_draw(letkf_ctx* c, unsigned long long frame, void* xi, void* v_out, cudaStream_t stream);
// The product part of noise_draw / draw_perturbations_on (normals already in xi).
int noise_product(letkf_ctx* c, const void* xi, void* v_out, cudaStream_t stream);
int draw_product_on(letkf_ctx* c, const void* xi, void* v_out, cudaStream_t stream);
int noise_normals_params(letkf_ctx* c, unsigned long long frame, void* xi, NormalsNode* nn);
int launch_copy_rows(letkf_ctx* c, const void* src, void* dst);

// fused.cu
// Host only: the fused kernel's shared-memory plan (c->fused_smem, c->dual) and SIMT threshold
// (c->simt_q, c->simt_ws) from the geometry, m, m_pad and simt_q_max; LETKF_EINVAL if it does not fit.
int fused_plan(letkf_ctx* c);
int fused_prepare(letkf_ctx* c);
int fused_step(letkf_ctx* c, const void* y, double sigma, void* xpred, int with_forecast);
// One launch of the fused kernel over the next frame of n systems (fused path, same device):
// their domains form one work queue (`queue`: 4 zeroed ints on the device, reset by the kernel).
constexpr int FUSED_MAX_BATCH = 32;
struct FusedFrame {
    letkf_ctx* c;
    const void* y;      // device slopes of the frame
    double sigma;       // <= 0: keep
    void* xpred;        // device prediction output, or null
    int with_forecast;
};
int fused_batch(const FusedFrame* f, int n, int* queue, cudaStream_t stream);
void fused_graph_reset(letkf_ctx* c);

}  // namespace letkf
