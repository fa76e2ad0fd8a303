// ppf_internal.h -- context layout and kernel launchers of the GB300 SIR filter.
#pragma once

#include <cstdint>
#include <cuda.h>  // CUtensorMap (the tensor map is encoded through the runtime's driver entry point)
#include <cuda_runtime.h>

#include "ppf.h"  // include/ppf.h (the build passes -I include)

#include <nvtx3/nvToolsExt.h>  // header-only; ranges cost nothing without an attached profiler

namespace ppf {

// A named NVTX range around one ABI call (visible in profiler timelines).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int TILE = 4096;          // particles per resampling tile (256 threads x 16)
constexpr int TILE_THREADS = 256;
constexpr int TILE_ITEMS = TILE / TILE_THREADS;
constexpr int ITEM_TICKETS = 8192;  // tickets per fill work item
constexpr int COPY_CHUNK = 8192;    // slots per routing-copy work item
constexpr int MAX_RADIUS = 8;
constexpr int MAX_SCHED_GROUPS = 16384;
// A proportional draw (systematic, RPA) with N_eff below N / BIN_CONCENTRATE
// fills every warp of 32 consecutive slots with the children of one or two
// parents, so the next step reads coherent patches whatever the spread
// before the draw: the resampling then sets the next step to the direct path.
constexpr double BIN_CONCENTRATE = 64.0;
constexpr int SCAN_SMEM_TILES = 16384;  // tile scan in shared memory up to this many tiles (N <= 67 M)
constexpr int BIN_MAX_BINS = 3073;      // binned likelihood: at most this many bins (tiles + 1)

// How the next step forms a slot's starting log-weight.
enum StepMode : int {
    MODE_CARRY = 0,     // identity ancestry, weight carried (no resampling since the last step)
    MODE_UNIFORM = 1,   // resampled: equal weights (lw_prev = 0)
    MODE_EXPLICIT = 2   // resampled: per-slot lw_prev buffer (RNA, restarts)
};

enum : int {
    FLAG_DEGENERATE = 1, FLAG_TIMEOUT = 2, FLAG_INTERNAL = 4, FLAG_BAD_ANCESTOR = 8, FLAG_KEPT = 16,
    FLAG_RING = 32  // ARNA redrew its ring
};

// per-block weight statistics of one step (online log-sum-exp partials)
struct Partial {
    float m, s0, s[5], s2, mp, sp;
};

// per-block statistics of one gradient step: log-sum-exp of l and the
// weighted sums of dl/d(sigma_PSF, A, I_bg, sigma_m)
struct GradPartial {
    float m, s0, s[4];
};

// device-side per-frame results and resampling scalars
struct DevSummary {
    double mean[5];
    double log_evidence;
    double ess;
    double max_lw;
    double log_total;          // M + log sum e^(lw - M), FP64
    float M;                   // max lw (exact float): the quantiser reference
    int32_t frame;
    int32_t flags;             // sticky FLAG_* bits, cleared by ppf_estimate
    int32_t degenerate;        // last resample kept every particle (no usable weight, or N_eff test)
    int64_t links, moved, max_group, min_group;
    uint64_t Q, u;             // last global resample: total fixed-point weight, offset
    uint64_t qN;               // and Q = qN N + qR (the ticket spacing in whole and remainder)
    uint32_t qR;
    int32_t n_items;           // fill work items of the last resample
    int32_t n_chunks;          // routing-copy work items of the last RPA resample
    int64_t mig;               // RNA: slots migrating to the next group
    int32_t involved;          // ARNA: groups that proportional allocation gives at least their size
    uint32_t blocks_done;      // step kernel: blocks that published partials
    double grad_L;             // ppf_loglik_grad: running sum of log-evidences
    double grad_g[4];          // and of their derivatives
    // likelihood path: bin_this is the path of the current step (set by the
    // frame preparation from bin_next or the caller's choice); bin_next is
    // decided by the step's finaliser from the warps it saw spread
    int32_t bin_this, bin_next;
    uint32_t spread_warps, total_warps;
    uint32_t bin_blocks_done;  // binned path: scatter blocks that finished
    int32_t n_bin_items;       // binned path: likelihood work items of this step
    int32_t n_split;           // two-stage RPA: extra work items of large or heavy groups (group_grid_kernel)
    int32_t n_runs;            // and the further runs of heavy tile parts, listed after them (split_runs_kernel)
    int32_t n_extra;           // the fill's further runs of ticket-heavy tiles (tile_tickets_kernel)
};

// two-stage RPA: one group's own systematic draw and where its offspring go
// (see group_grid_kernel), read by the group's block as six 16-byte loads
struct alignas(16) GroupGrid {
    uint64_t Ca;     // cumulative fixed-point weight below the group
    uint64_t Q;      // the group's total
    uint64_t u;      // its ticket offset
    uint64_t qN;     // Q = qN nt + qR
    uint64_t dm;     // floor((2^64 - 1) / nt)
    int64_t p0, p1;  // its particles [p0, p1)
    int64_t tg0;     // its first ticket slot in the global ticket order
    int64_t keep;    // its offspring that stay (GS, SGS: min(nt, n_g))
    int64_t shift;   // the slot of its first kept offspring (the balanced offset)
    uint32_t qR;
    uint32_t nt;     // its offspring count (0: nothing to draw)
};

struct Scratch {
    uint64_t *Qt;      // [T]   tile totals
    uint64_t *Ct;      // [T+1] exclusive tile prefix
    int64_t *Tt;       // [T+1] tickets below each tile start
    int32_t *item_off; // [T+1] fill work-item prefix per tile
    int32_t *extra;    // [2 (N / ITEM_TICKETS + 1)] the fill's further runs (tile, run) of ticket-heavy tiles
    uint64_t *Cbl;     // [G+1] local prefix at group starts (within their tile)
    int64_t *Tg;       // [G+1] tickets below each group start
    int32_t *tile_g;   // [2T] per tile: first group starting at or after it, group starts inside (capped)
    GroupGrid *ggrid;  // [G]  two-stage RPA: every group's draw
    int32_t *split;    // [4 (T + G + 2 N / ITEM_TICKETS + 2)] two-stage RPA: extra work items (tile or -1, group, run, 0)
    // scheduler (RPA)
    uint64_t *skey;    // [2G] sort / merge buffers
    int64_t *sval;     // [5G]
    int32_t *seg_src;  // segments: ticket start, slot start, length, chunk prefix
    int64_t *seg_tick;
    int64_t *seg_dst;
    int64_t *seg_len;
    int32_t *seg_chunk; // [2G+1]
};

}  // namespace ppf

struct ppf_ctx {
    ppf_model m;
    int64_t N;
    int32_t group_size, G, T;     // groups, resampling tiles
    cudaStream_t stream;
    cudaStream_t side_stream;     // the RPA schedule, concurrent with the fill
    cudaEvent_t ev_scan, ev_sched;  // fork after the tile scan, join before the routing copy
    int device, num_sms;
    float *state[2];              // 6 x N SoA each
    int cur;                      // index of the current particles
    int32_t *anc;                 // pending ancestors
    int32_t *anc_sys;             // systematic ancestors before RPA routing
    float *lwp;                   // per-slot starting log-weights (MODE_EXPLICIT)
    int64_t *goff, *goff_new;     // group offsets [G+1]
    int32_t *ring, *succ;         // ARNA ring order [G] and each group's successor on it [G]
    float *Zp;                    // padded frame minus background
    float2 *lmap;                 // pcSIR: (B, C) patch sums of every anchor (W + 2r) x (H + 2r)
    int32_t Wp, Hp, pad;
    void *frame_buf[2];           // device copies for ppf_step_host (double-buffered)
    int fb_next;                  // buffer the next ppf_step_host fills
    bool fb_used[2];
    cudaStream_t copy_stream;     // host-to-device frame copies, overlapping the previous frame
    cudaEvent_t fb_copied[2], fb_free[2];
    size_t frame_bytes;
    ppf::Partial *part;
    int n_part;
    float *tang[2];               // gradient: d(x, y)/dsigma_m tangents, 2 x N each
    int tcur;
    ppf::GradPartial *gpart;
    ppf::DevSummary *sum;
    ppf::DevSummary *sum_host;    // pinned mirror for ppf_estimate
    ppf_estimate_t *est_dev;      // device staging of ppf_estimate_async
    ppf::Scratch sc;
    // binned likelihood path (input-space decomposition): tiles of bin_T
    // anchors, bin_nbins bins (the last for particles with no patch sum)
    int32_t bin_T, bin_nx, bin_nbins, bin_grid, bin_items_max;  // bin_grid: blocks of the binned likelihood
    int bin_force;                // -1: chosen per step on the device; 0: direct path; 1: binned path
    uint32_t *bin_key;            // [N] bin of every slot, then the place of its record in bin order
    uint32_t *bin_tot;            // [2 (nbins + 1)] bin sizes, then the scatter's cursors (offsets inside each bin)
    int32_t *bin_item;            // [3 x items_max] work items: bin, first record, count
    float4 *bin_rec;              // [N] records in bin order: (x, y, I0, -)
    float *bin_l;                 // [N] l of every record, in bin order
    CUtensorMap bin_tmap;         // the prepared frame as a 2D float tensor for the window copies (64-byte aligned type)
    int mode;                     // StepMode of the next step
    bool stepped;                 // at least one step since create/set
    bool weighted;                // a step happened since the last resample
    int32_t last_frame;
    // profiling (ppf_profile_enable)
    bool prof_on;
    int32_t prof_cap;
    cudaEvent_t *prof_ev;         // [4 phases][cap][2]
    int32_t prof_n[4];
    int64_t launches, n_steps, n_resamples, h2d_bytes, d2h_bytes;
    char err[512];
};

namespace ppf {
enum Phase { PH_PREPARE = 0, PH_STEP = 1, PH_FINALIZE = 2, PH_RESAMPLE = 3 };

// A launch that the GPU may schedule while the previous kernel of the stream
// is still running (programmatic dependent launch): the kernel must execute
// pdl_wait() before it reads anything the previous kernel writes, and before
// it returns, so that kernels launched after it still see every earlier one
// complete.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}
// record the start / end event of a phase when profiling is on
void prof_mark(ppf_ctx *c, int phase, int end);
// launchers (each enqueues on ctx->stream; return cudaGetLastError())
cudaError_t launch_init(ppf_ctx *c);
cudaError_t launch_prepare_frame(ppf_ctx *c, const void *frame);
cudaError_t launch_step(ppf_ctx *c, int32_t k);
cudaError_t launch_grad_step(ppf_ctx *c, int32_t k, bool first, int32_t *anchors);
cudaError_t resample_kernel_attributes();
cudaError_t launch_resample_global(ppf_ctx *c, int scheme, double ess_thr);
cudaError_t launch_resample_rna(ppf_ctx *c, float alpha, double ess_thr);
cudaError_t launch_resample_arna(ppf_ctx *c, float alpha, double ess_thr);
cudaError_t launch_identity(ppf_ctx *c, int32_t *dst);
cudaError_t launch_pending(ppf_ctx *c, int32_t *anc_out, float *lwp_out);
cudaError_t launch_fill_f32(ppf_ctx *c, float *dst, float v);
cudaError_t launch_format_estimate(ppf_ctx *c);
cudaError_t launch_cell_map(ppf_ctx *c);
int step_grid(ppf_ctx *c);
// binned likelihood path (ppf_binned.cu)
cudaError_t bin_setup(ppf_ctx *c);                      // tile geometry, buffers and tensor map (at create)
cudaError_t launch_binned(ppf_ctx *c);                  // scatter and likelihood (exit early when not chosen)
cudaError_t bin_set_next(ppf_ctx *c, int binned);       // the path of the next step in auto mode
}  // namespace ppf
