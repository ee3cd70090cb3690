// Host-side context of one lattice and the internal launch interface between
// the C-ABI layer (lbm_api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include <type_traits>

#include "lbm_cell.cuh"

struct lbm_ctx {
    lbm_params p;
    double rho_held[2][2];       // densities (A, B) of the inlet [0] and outlet [1] cells
    long long n_held = 0;        // number of inlet / outlet cells in the geometry
    double mss = 0.0;            // mass-sink-source rate (lbm_set_mss)
    struct lbm_batch *owner = nullptr;  // the batch of a view
    int dev = 0;
    cudaStream_t stream = nullptr;
    int n = 0;
    lbm::DevParams dp{};
    lbm_constitutive curves[LBM_MAX_PORE_TYPES];

    // device buffers (owned)
    float *f[2] = {nullptr, nullptr};  // populations [2][19][n] (F32 or 16-bit slots), ping-pong
    int cur = 0;                       // buffer holding the latest state
    uint8_t *type = nullptr;           // [n]
    float *phi = nullptr;              // [n] porosity (1 pore, 0 solid)
    lbm::GrayRec *gray = nullptr;      // [n], valid at gray cells only
    float *rho = nullptr;              // [2][n] densities of the current step
    float *rho_cap = nullptr;          // [3][n]: while set, fused steps also store their densities there
    float *macro = nullptr;            // [6][n] rhoA, rhoB, ux, uy, uz, Sw
    double *red = nullptr;             // reduction partials
    int red_blocks = 0;
    // published-density march (lbm_march.cu)
    uint32_t *wmask = nullptr;         // [n] static wall mask: bits 1..18 neighbour solid/outside, 24..31 type
    float2 *pub = nullptr;             // [n] densities (drho^A, drho^B) published during a step
    unsigned *prog = nullptr;          // [prog_len] error flag, finished CTAs, progress per work item
    int prog_len = 0;

    int path = 0;   // 0: fused single launch, 1: two launches (density, collide)
    int tile = 8;   // fused tile variant (lbm_set_kernel); 8 = automatic among 2, 4, 7; 5, 6 = the march
    int auto_tile = -1;  // the automatic choice, once made (depends on the grid only)
    bool has_geometry = false;
    bool has_fields = false;
    bool view = false;  // a run of a batch: buffers owned by the batch
    long long steps = 0;
    long long launches = 0;

    // CUDA-graph replay of runs of steps on small lattices (launch-bound):
    // one executable graph per buffer parity, each GRAPH_STEPS steps without
    // field output; dropped whenever a parameter the kernels take by value
    // changes
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long long graph_launches = 0;  // kernel launches one replay stands for
    cudaStream_t cap = nullptr;    // private capture stream
    bool graph_off = false;        // a capture failed: step directly from then on

    struct ProfRec {
        const char *name;
        cudaEvent_t a, b;
    };
    bool profiling = false;
    std::vector<ProfRec> prof;

    int fail_launches = 0;  // step launches still to be issued with an invalid shape (lbm_inject_launch_failures)
};

namespace lbm {

// Observables reduction: blocks of the partial sums for n cells, and the
// number of FP64 values it returns.
int obs_blocks(int n);
constexpr int NOBS_HOST = 16;

// A run of the batch changed a per-run parameter: its next step re-reads the runs.
void batch_runs_changed(struct lbm_batch *b);

// Steps per replayed graph (even: the replay returns to the same buffer) and
// the largest lattice that replays graphs (above it a step is long enough to
// hide its launch).
constexpr int GRAPH_STEPS = 32;
constexpr int GRAPH_MAX_CELLS = 1 << 18;
// Frees the context's step graphs (the next lbm_step captures new ones).
void drop_graphs(lbm_ctx *ctx);

// Kernel launches (each records itself in ctx->launches and, while profiling,
// brackets the launch with CUDA events).
cudaError_t launch_init(lbm_ctx *ctx, const float *rhoA, const float *rhoB, const float *u);
cudaError_t launch_density(lbm_ctx *ctx);
cudaError_t launch_collide(lbm_ctx *ctx, bool write_macro);
cudaError_t launch_fused(lbm_ctx *ctx, bool write_macro);
// The fused tile a step of ctx runs: the requested one, with tile 8 resolved
// to its per-grid choice and the shapes a storage does not have mapped to 2
// (the shifted 16-bit kernel has 32x8 and 64x7).
int fused_tile_in_use(lbm_ctx *ctx);
// The published-density march (tiles 5 and 6); *ran false where it does not apply.
cudaError_t launch_march(lbm_ctx *ctx, bool write_macro, bool *ran);
cudaError_t launch_wallmask(lbm_ctx *ctx);
// Reads and clears the march's wait-timeout flag (synchronises the stream).
cudaError_t march_take_error(lbm_ctx *ctx, int *flag);
constexpr int MARCH_PROG_LEN = 2 + 4096;  // error flag, finished count, work items
cudaError_t launch_fused_lp(lbm_ctx *ctx, bool write_macro);
cudaError_t launch_d2q9_init(lbm_ctx *ctx, const float *rhoA, const float *rhoB, const float *u);
cudaError_t launch_d2q9_step(lbm_ctx *ctx, bool write_macro);
cudaError_t launch_geometry(lbm_ctx *ctx, const uint8_t *ptype);
cudaError_t launch_observables(lbm_ctx *ctx, double *host_out16);
// The same without the final synchronisation (the copy is left in flight).
cudaError_t launch_observables(lbm_ctx *ctx, double *host_out16, bool sync);
cudaError_t launch_static_out(lbm_ctx *ctx, float *kinv6, float *pcs, float *swirr, float *sores);

// Rest-referenced 16-bit layout views of population buffers bi (in) and bo
// (out): int32 rest populations [2][n] first, then the 16-bit slots.
template <class LY>
inline LY lay_r16(lbm_ctx *ctx, int bi, int bo)
{
    return LY::make(ctx->f[bi], ctx->f[bo], ctx->n);
}

// Block shape of a step launch: threads, or a zero-size block (a
// configuration the CUDA runtime rejects on the host, before any device work)
// while lbm_inject_launch_failures has launches pending.  Every step launcher
// checks the launch before it counts it or flips the buffer parity.
inline dim3 step_block(lbm_ctx *ctx, int threads)
{
    if (ctx->fail_launches > 0) {
        --ctx->fail_launches;
        return dim3(0, 1, 1);
    }
    return dim3(threads, 1, 1);
}

// Profiling helpers used around launches.
void prof_begin(lbm_ctx *ctx, const char *name, cudaEvent_t *ev_out);
void prof_end(lbm_ctx *ctx, const char *name, cudaEvent_t ev_begin);

}  // namespace lbm
