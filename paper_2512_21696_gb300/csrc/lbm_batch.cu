// Batched lattices (REV library runs of the workflow's step ii): many
// independent lattices of uneven size advanced together.
//
//   * one persistent launch per step and tile shape (k_fused_batch): CTAs
//     take (run, column, z-chunk) items from a global counter, largest runs
//     first, so uneven sizes balance without any waiting;
//   * k steps are captured once into a CUDA graph (counter resets and
//     launches) and replayed;
//   * lbm_batch_tune times every candidate tile shape on the runs of each
//     x-extent and keeps the fastest per extent (runs whose best shapes
//     differ are stepped by one launch per shape);
//   * every run is also an ordinary context ("view") over its slice of the
//     batch buffers, so geometry, fields, observables and checkpoints of a
//     run use the single-lattice calls.
// All per-cell arithmetic is the single-lattice kernel's (lbm_fused.cuh): a
// run advanced in a batch is bit-identical to the run advanced alone.
#include <algorithm>
#include <cmath>
#include <map>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_fused.cuh"
#include "lbm_host.h"

using namespace lbm_host;

namespace lbm {

// Batched step: the work items of many lattices (runs) in one persistent
// launch.  CTAs take items from a global counter (one atomic per item, no
// waiting), largest runs first; an item is (run, column, z-chunk).  Each run
// is a self-contained lattice whose slots, cell types, gray records and
// fields sit at its own offsets of the batch buffers.
template <int TX, int TY, int MINB, bool MACRO, bool EXT, class LY>
__global__ void __launch_bounds__(TX *TY, MINB)
    k_fused_batch(DevParams P, const BatchRun *__restrict__ runs, int nruns, int nitems,
                  unsigned int *__restrict__ counter, const unsigned char *__restrict__ fin,
                  unsigned char *__restrict__ fout, const uint8_t *__restrict__ type, GrayRec *__restrict__ gray,
                  float *__restrict__ macro)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nitems) return;
        int lo = 0, hi = nruns - 1;  // last run with item0 <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (runs[mid].item0 <= item) lo = mid; else hi = mid - 1;
        }
        const BatchRun R = runs[lo];
        Geo G;
        G.nx = R.nx;
        G.ny = R.ny;
        G.nz = R.nz;
        G.n = R.n;
        for (int a = 0; a < 2; ++a)
            for (int d = 0; d < 3; ++d) G.accel[a][d] = R.accel[a][d];
        for (int k = 0; k < 8; ++k) (&G.held[0][0][0])[k] = (&R.held[0][0][0])[k];
        G.mss = R.mss;
        const int local = item - R.item0;
        const int col = local % R.ncol, chunk = local / R.ncol;
        const int za = (int)((long long)R.nz * chunk / R.zchunks);
        const int zb = (int)((long long)R.nz * (chunk + 1) / R.zchunks);
        if (za >= zb) continue;
        const LY ly = LY::make(fin + R.pop_off, fout + R.pop_off, R.n);
        fused_item<TX, TY, MACRO, EXT>(P, G, ly, type + R.cell_off, gray + R.cell_off, macro + 6 * R.cell_off,
                                  (col % R.tiles_x) * TX, (col / R.tiles_x) * TY, za, zb, smem_raw);
    }
}

}  // namespace lbm

namespace {

// Tile shapes of the batch kernel.
struct TileShape {
    int tx, ty, minb;
};
constexpr TileShape BATCH_TILES[] = {{32, 8, 2}, {16, 16, 2}, {32, 16, 1}};
constexpr int N_BATCH_TILES = 3;

template <int TX, int TY, int MINB, bool MACRO, bool EXT, class LY>
cudaError_t prep_kernel(int *slots, int dev)
{
    auto kern = lbm::k_fused_batch<TX, TY, MINB, MACRO, EXT, LY>;
    const size_t smem = lbm::Tiles<TX, TY>::smem();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * TY, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    *slots = std::max(per_sm, 1) * sms;
    return cudaSuccess;
}

}  // namespace

struct lbm_batch {
    int dev = 0;
    cudaStream_t stream = nullptr;
    lbm_params p0;  // run 0's parameters (the shared physics)
    std::vector<lbm_ctx *> views;
    std::vector<long long> cell_off, pop_off;
    long long cells = 0;
    size_t pop_total = 0;
    void *f[2] = {nullptr, nullptr};
    uint8_t *type = nullptr;
    float *phi = nullptr;
    lbm::GrayRec *gray = nullptr;
    float *rho = nullptr;
    float *macro = nullptr;
    double *red = nullptr;
    int cur = 0;
    long long steps = 0, launches = 0;
    std::vector<int> tile_of_run;  // index into BATCH_TILES
    struct Group {
        int tile;
        std::vector<int> runs;
        std::vector<lbm::BatchRun> host;  // the item table as uploaded (runs in the order above)
        lbm::BatchRun *d_runs = nullptr;
        unsigned int *counter = nullptr;
        int nruns = 0, nitems = 0, grid = 0;
    };
    std::vector<Group> groups;
    bool groups_ok = false;
    bool ext = false;         // some run has reservoir cells or a mass-sink-source rate
    bool runs_dirty = false;  // a run's reservoir densities or rate changed since the upload
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // (steps, parity)
    cudaStream_t cap = nullptr;  // private stream the graphs are captured on
};

namespace {

void free_groups(lbm_batch *b)
{
    for (auto &g : b->groups) {
        cudaFree(g.d_runs);
        cudaFree(g.counter);
    }
    b->groups.clear();
    b->groups_ok = false;
}
void free_graphs(lbm_batch *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// Work items of one run for a tile shape: columns x z-chunks of `planes`
// planes (the z-march amortises its two halo planes over them).
lbm::BatchRun describe_run(const lbm_batch *b, int r, const TileShape &ts, int planes)
{
    const lbm_params &p = b->views[r]->p;
    lbm::BatchRun R{};
    R.nx = p.nx;
    R.ny = p.ny;
    R.nz = p.nz;
    R.n = b->views[r]->n;
    R.tiles_x = (p.nx + ts.tx - 1) / ts.tx;
    R.ncol = R.tiles_x * ((p.ny + ts.ty - 1) / ts.ty);
    R.zchunks = std::max(1, (p.nz + planes / 2) / planes);
    R.cell_off = b->cell_off[r];
    R.pop_off = b->pop_off[r];
    for (int a = 0; a < 2; ++a)
        for (int d = 0; d < 3; ++d) R.accel[a][d] = (float)p.body_accel[a][d];
    for (int k = 0; k < 8; ++k) (&R.held[0][0][0])[k] = (&b->views[r]->dp.held[0][0][0])[k];
    R.mss = b->views[r]->dp.mss;
    return R;
}

int slots_for(const lbm_batch *b, int tile, int *slots);

// Builds the item tables of the groups (one per tile shape in use).
int build_groups(lbm_batch *b, const std::vector<int> &subset, const std::vector<int> &tile_of_run)
{
    free_groups(b);
    std::map<int, std::vector<int>> by_tile;
    for (int r : subset) by_tile[tile_of_run[r]].push_back(r);
    for (auto &kv : by_tile) {
        lbm_batch::Group g;
        g.tile = kv.first;
        g.runs = kv.second;
        std::sort(g.runs.begin(), g.runs.end(), [&](int x, int y) { return b->views[x]->n > b->views[y]->n; });
        int slots = 0;
        const int rc = slots_for(b, g.tile, &slots);
        if (rc != LBM_OK) return rc;
        // planes per item: up to 16, fewer when the group has too little work
        // for about four items per resident CTA (small batches, small runs)
        const TileShape &ts = BATCH_TILES[g.tile];
        long long colplanes = 0;
        for (int r : g.runs) {
            const lbm_params &p = b->views[r]->p;
            colplanes += (long long)((p.nx + ts.tx - 1) / ts.tx) * ((p.ny + ts.ty - 1) / ts.ty) * p.nz;
        }
        const int planes = (int)std::max(1LL, std::min(16LL, colplanes / (4LL * slots)));
        std::vector<lbm::BatchRun> host;
        int items = 0;
        for (int r : g.runs) {
            lbm::BatchRun R = describe_run(b, r, ts, planes);
            R.item0 = items;
            items += R.ncol * R.zchunks;
            host.push_back(R);
        }
        g.nruns = (int)host.size();
        g.nitems = items;
        g.grid = std::max(1, std::min(items, slots));
        LBM_CUDA(cudaMalloc(&g.d_runs, host.size() * sizeof(lbm::BatchRun)));
        LBM_CUDA(cudaMalloc(&g.counter, sizeof(unsigned int)));
        LBM_CUDA(cudaMemcpyAsync(g.d_runs, host.data(), host.size() * sizeof(lbm::BatchRun),
                                 cudaMemcpyHostToDevice, b->stream));
        g.host = std::move(host);
        b->groups.push_back(std::move(g));
    }
    LBM_CUDA(cudaStreamSynchronize(b->stream));
    b->groups_ok = true;
    return LBM_OK;
}

template <int TX, int TY, int MINB, class LY>
cudaError_t launch_group_t(lbm_batch *b, const lbm_batch::Group &g, bool macro)
{
    const size_t smem = lbm::Tiles<TX, TY>::smem();
    const unsigned char *fin = reinterpret_cast<const unsigned char *>(b->f[b->cur]);
    unsigned char *fout = reinterpret_cast<unsigned char *>(b->f[1 - b->cur]);
    cudaError_t e = cudaMemsetAsync(g.counter, 0, sizeof(unsigned int), b->stream);
    if (e != cudaSuccess) return e;
    const lbm::DevParams &P = b->views[0]->dp;
    auto kern = macro ? (b->ext ? lbm::k_fused_batch<TX, TY, MINB, true, true, LY>
                                : lbm::k_fused_batch<TX, TY, MINB, true, false, LY>)
                      : (b->ext ? lbm::k_fused_batch<TX, TY, MINB, false, true, LY>
                                : lbm::k_fused_batch<TX, TY, MINB, false, false, LY>);
    kern<<<g.grid, TX * TY, smem, b->stream>>>(P, g.d_runs, g.nruns, g.nitems, g.counter, fin, fout, b->type,
                                               b->gray, b->macro);
    return cudaGetLastError();
}

template <int TX, int TY, int MINB>
cudaError_t launch_group_s(lbm_batch *b, const lbm_batch::Group &g, bool macro)
{
    switch (b->p0.storage) {
    case LBM_STORAGE_F16R: return launch_group_t<TX, TY, MINB, lbm::LayF16R>(b, g, macro);
    case LBM_STORAGE_BF16R: return launch_group_t<TX, TY, MINB, lbm::LayB16R>(b, g, macro);
    default: return launch_group_t<TX, TY, MINB, lbm::LayF32>(b, g, macro);
    }
}

cudaError_t launch_group(lbm_batch *b, const lbm_batch::Group &g, bool macro)
{
    switch (g.tile) {
    case 1: return launch_group_s<16, 16, 2>(b, g, macro);
    case 2: return launch_group_s<32, 16, 1>(b, g, macro);
    default: return launch_group_s<32, 8, 2>(b, g, macro);
    }
}

template <int TX, int TY, int MINB, class LY>
cudaError_t prep_t(int *slots, int dev)
{
    cudaError_t e = prep_kernel<TX, TY, MINB, true, false, LY>(slots, dev);
    if (e == cudaSuccess) e = prep_kernel<TX, TY, MINB, false, false, LY>(slots, dev);
    if (e == cudaSuccess) e = prep_kernel<TX, TY, MINB, true, true, LY>(slots, dev);
    if (e != cudaSuccess) return e;
    return prep_kernel<TX, TY, MINB, false, true, LY>(slots, dev);
}
template <int TX, int TY, int MINB>
cudaError_t prep_s(const lbm_batch *b, int *slots)
{
    switch (b->p0.storage) {
    case LBM_STORAGE_F16R: return prep_t<TX, TY, MINB, lbm::LayF16R>(slots, b->dev);
    case LBM_STORAGE_BF16R: return prep_t<TX, TY, MINB, lbm::LayB16R>(slots, b->dev);
    default: return prep_t<TX, TY, MINB, lbm::LayF32>(slots, b->dev);
    }
}
int slots_for(const lbm_batch *b, int tile, int *slots)
{
    cudaError_t e;
    switch (tile) {
    case 1: e = prep_s<16, 16, 2>(b, slots); break;
    case 2: e = prep_s<32, 16, 1>(b, slots); break;
    default: e = prep_s<32, 8, 2>(b, slots); break;
    }
    return e == cudaSuccess ? LBM_OK : cuda_fail(e, "batch kernel setup");
}

// Picks the march for the runs (with reservoir cells or a mass-sink-source
// rate, or neither; a change drops the captured graphs) and uploads per-run
// parameters changed since the item tables were built.  The graphs read the
// tables from device memory, so an upload needs no new capture.
int sync_runs(lbm_batch *b)
{
    // the kernel reads the curve table of run 0 for every run
    const lbm_ctx *v0 = b->views[0];
    for (const auto *v : b->views)
        if (std::memcmp(v->curves, v0->curves, sizeof(v0->curves)) != 0) return LBM_ERR_STATE;
    bool ext = false;
    for (auto *v : b->views) ext = ext || v->n_held > 0 || v->mss != 0.0;
    if (ext != b->ext) {
        b->ext = ext;
        free_graphs(b);
    }
    if (b->runs_dirty && b->groups_ok) {
        for (auto &g : b->groups) {
            for (size_t k = 0; k < g.runs.size(); ++k) {
                const lbm::DevParams &dp = b->views[g.runs[k]]->dp;
                for (int q = 0; q < 8; ++q) (&g.host[k].held[0][0][0])[q] = (&dp.held[0][0][0])[q];
                g.host[k].mss = dp.mss;
            }
            LBM_CUDA(cudaMemcpyAsync(g.d_runs, g.host.data(), g.host.size() * sizeof(lbm::BatchRun),
                                     cudaMemcpyHostToDevice, b->stream));
        }
    }
    b->runs_dirty = false;
    return LBM_OK;
}

// nsteps steps of the current groups, enqueued on the stream.
int enqueue_steps(lbm_batch *b, int nsteps)
{
    for (int k = 0; k < nsteps; ++k) {
        for (const auto &g : b->groups) LBM_CUDA(launch_group(b, g, k == nsteps - 1));
        b->cur = 1 - b->cur;
    }
    return LBM_OK;
}

bool same_physics(const lbm_params &a, const lbm_params &b)
{
    for (int k = 0; k < 3; ++k)
        if (a.periodic[k] != b.periodic[k]) return false;
    for (int k = 0; k < 2; ++k)
        if (a.tau[k] != b.tau[k] || a.phi_avg[k] != b.phi_avg[k] || a.phi_max[k] != b.phi_max[k] ||
            a.rho_wall[k] != b.rho_wall[k])
            return false;
    return a.G == b.G && a.kappa_csf == b.kappa_csf && a.csf_everywhere == b.csf_everywhere &&
           a.wet_idx == b.wet_idx && a.rho_hi == b.rho_hi && a.rho_lo == b.rho_lo && a.s_lo == b.s_lo &&
           a.s_hi == b.s_hi && a.at_cut == b.at_cut && a.eps_n == b.eps_n && a.kr_min == b.kr_min &&
           a.c_g == b.c_g && a.storage == b.storage && a.stream == b.stream;
}

void sync_views(lbm_batch *b, int nsteps)
{
    for (auto *v : b->views) {
        v->cur = b->cur;
        v->steps += nsteps;
    }
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_batch **out, int nruns, const lbm_params *runs)
{
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (nruns < 1 || !runs) return LBM_ERR_ARG;
    for (int r = 0; r < nruns; ++r) {
        const int vr = validate_params(&runs[r]);
        if (vr != LBM_OK) return vr;
        if (!same_physics(runs[0], runs[r])) return LBM_ERR_ARG;
    }
    if (runs[0].storage == LBM_STORAGE_F16S || runs[0].storage == LBM_STORAGE_BF16S) return LBM_ERR_ARG;
    for (int r = 0; r < nruns; ++r)
        if (runs[r].lattice != LBM_LATTICE_D3Q19) return LBM_ERR_ARG;
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_OOM;
    b->p0 = runs[0];
    b->stream = (cudaStream_t)runs[0].stream;
    if (cudaGetDevice(&b->dev) != cudaSuccess) {
        delete b;
        return cuda_fail(cudaGetLastError(), "cudaGetDevice");
    }
    int max_n = 0;
    for (int r = 0; r < nruns; ++r) {
        lbm_ctx *v = new (std::nothrow) lbm_ctx();
        if (!v) {
            lbm_batch_destroy(b);
            return LBM_ERR_OOM;
        }
        v->p = runs[r];
        v->n = runs[r].nx * runs[r].ny * runs[r].nz;
        v->dev = b->dev;
        v->stream = b->stream;
        v->view = true;
        v->owner = b;
        for (int k = 0; k < LBM_MAX_PORE_TYPES; ++k) lbm_default_constitutive(&v->curves[k]);
        default_held(v);
        fill_device_params(v);
        b->views.push_back(v);
        b->cell_off.push_back(b->cells);
        b->pop_off.push_back((long long)b->pop_total);
        b->cells += v->n;
        b->pop_total += (pop_bytes(v) + 255) / 256 * 256;
        max_n = std::max(max_n, v->n);
    }
    b->tile_of_run.assign(nruns, 0);
    const size_t N = (size_t)b->cells;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMalloc(&b->f[k], b->pop_total);
        if (e == cudaSuccess) e = cudaMemset(b->f[k], 0, b->pop_total);  // solid cells' slots stay zero
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->type, N);
    if (e == cudaSuccess) e = cudaMalloc(&b->phi, N * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b->gray, N * sizeof(lbm::GrayRec));
    if (e == cudaSuccess) e = cudaMalloc(&b->rho, 3 * N * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b->macro, 6 * N * sizeof(float));
    const int red_blocks = lbm::obs_blocks(max_n);
    if (e == cudaSuccess) e = cudaMalloc(&b->red, (size_t)(red_blocks + 1) * lbm::NOBS_HOST * sizeof(double));
    // zero: the reduction's completion count starts there
    if (e == cudaSuccess) e = cudaMemset(b->red, 0, (size_t)(red_blocks + 1) * lbm::NOBS_HOST * sizeof(double));
    if (e != cudaSuccess) {
        const int code = cuda_fail(e, "lbm_batch_create allocation");
        lbm_batch_destroy(b);
        return code;
    }
    for (int r = 0; r < nruns; ++r) {
        lbm_ctx *v = b->views[r];
        const size_t co = (size_t)b->cell_off[r];
        for (int k = 0; k < 2; ++k) v->f[k] = reinterpret_cast<float *>(reinterpret_cast<char *>(b->f[k]) + b->pop_off[r]);
        v->type = b->type + co;
        v->phi = b->phi + co;
        v->gray = b->gray + co;
        v->rho = b->rho + 3 * co;
        v->macro = b->macro + 6 * co;
        v->red = b->red;
        v->red_blocks = lbm::obs_blocks(v->n);
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return LBM_OK;
    DeviceGuard g(b->dev);
    free_graphs(b);
    free_groups(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (auto *v : b->views) delete v;
    cudaFree(b->f[0]);
    cudaFree(b->f[1]);
    cudaFree(b->type);
    cudaFree(b->phi);
    cudaFree(b->gray);
    cudaFree(b->rho);
    cudaFree(b->macro);
    cudaFree(b->red);
    delete b;
    return LBM_OK;
}

int lbm_batch_run(lbm_batch *b, int run, lbm_ctx **view)
{
    if (!b || !view || run < 0 || run >= (int)b->views.size()) return LBM_ERR_ARG;
    *view = b->views[run];
    return LBM_OK;
}

int lbm_batch_step(lbm_batch *b, int nsteps)
{
    if (!b || nsteps < 0) return LBM_ERR_ARG;
    for (auto *v : b->views)
        if (!v->has_fields || v->cur != b->cur) return LBM_ERR_STATE;
    if (nsteps == 0) return LBM_OK;
    DeviceGuard dg(b->dev);
    if (!dg.ok) return LBM_ERR_CUDA;
    int src = sync_runs(b);
    if (src != LBM_OK) return src;
    if (!b->groups_ok) {
        std::vector<int> all(b->views.size());
        for (size_t r = 0; r < all.size(); ++r) all[r] = (int)r;
        const int rc = build_groups(b, all, b->tile_of_run);
        if (rc != LBM_OK) return rc;
        free_graphs(b);
    }
    const auto key = std::make_pair(nsteps, b->cur);
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        // capture on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); the graph is launched on the
        // caller's stream
        if (!b->cap) LBM_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        const int cur0 = b->cur;
        cudaGraph_t graph = nullptr;
        const cudaStream_t user = b->stream;
        b->stream = b->cap;
        cudaError_t be = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        const int rc = be == cudaSuccess ? enqueue_steps(b, nsteps) : cuda_fail(be, "cudaStreamBeginCapture");
        const cudaError_t ce = be == cudaSuccess ? cudaStreamEndCapture(b->cap, &graph) : cudaSuccess;
        b->stream = user;
        b->cur = cur0;
        if (rc != LBM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate");
        it = b->graphs.emplace(key, exec).first;
    }
    LBM_CUDA(cudaGraphLaunch(it->second, b->stream));
    b->cur = (b->cur + nsteps) & 1;
    b->steps += nsteps;
    b->launches += (long long)nsteps * (long long)b->groups.size();
    sync_views(b, nsteps);
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch *b, int trial_steps, int *tiles_out)
{
    if (!b || trial_steps < 2) return LBM_ERR_ARG;
    for (auto *v : b->views)
        if (!v->has_fields || v->cur != b->cur) return LBM_ERR_STATE;
    DeviceGuard dg(b->dev);
    if (!dg.ok) return LBM_ERR_CUDA;
    const int src = sync_runs(b);
    if (src != LBM_OK) return src;
    trial_steps += trial_steps & 1;  // even: the buffer parity returns
    // save the state the trials advance (populations, residual flags, fields)
    const size_t gray_bytes = (size_t)b->cells * sizeof(lbm::GrayRec), macro_bytes = 6 * (size_t)b->cells * 4;
    void *save_f = nullptr, *save_gray = nullptr, *save_macro = nullptr;
    cudaError_t e = cudaMalloc(&save_f, b->pop_total);
    if (e == cudaSuccess) e = cudaMalloc(&save_gray, gray_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&save_macro, macro_bytes);
    if (e != cudaSuccess) {
        cudaFree(save_f);
        cudaFree(save_gray);
        cudaFree(save_macro);
        return cuda_fail(e, "lbm_batch_tune allocation");
    }
    e = cudaMemcpyAsync(save_f, b->f[b->cur], b->pop_total, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(save_gray, b->gray, gray_bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(save_macro, b->macro, macro_bytes, cudaMemcpyDeviceToDevice, b->stream);
    // classes of runs by x extent (the extent that decides lane use)
    std::map<int, std::vector<int>> classes;
    for (size_t r = 0; r < b->views.size(); ++r) classes[b->views[r]->p.nx].push_back((int)r);
    std::vector<int> best(b->views.size(), 0);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    int rc = e == cudaSuccess ? LBM_OK : cuda_fail(e, "lbm_batch_tune setup");
    for (auto it = classes.begin(); rc == LBM_OK && it != classes.end(); ++it) {
        float best_ms = 0.f;
        int best_tile = 0;
        for (int t = 0; t < N_BATCH_TILES && rc == LBM_OK; ++t) {
            std::vector<int> tiles(b->views.size(), t);
            rc = build_groups(b, it->second, tiles);
            if (rc != LBM_OK) break;
            rc = enqueue_steps(b, 2);  // warm-up
            if (rc == LBM_OK && cudaEventRecord(t0, b->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
            if (rc == LBM_OK) rc = enqueue_steps(b, trial_steps);
            if (rc == LBM_OK && cudaEventRecord(t1, b->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
            if (rc == LBM_OK && cudaEventSynchronize(t1) != cudaSuccess) rc = LBM_ERR_CUDA;
            float ms = 0.f;
            if (rc == LBM_OK && cudaEventElapsedTime(&ms, t0, t1) != cudaSuccess) rc = LBM_ERR_CUDA;
            if (rc == LBM_OK && (t == 0 || ms < best_ms)) {
                best_ms = ms;
                best_tile = t;
            }
        }
        for (int r : it->second) best[r] = best_tile;
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    // restore the state (the trials took an even number of steps)
    if (rc == LBM_OK) {
        e = cudaMemcpyAsync(b->f[b->cur], save_f, b->pop_total, cudaMemcpyDeviceToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->gray, save_gray, gray_bytes, cudaMemcpyDeviceToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->macro, save_macro, macro_bytes, cudaMemcpyDeviceToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "lbm_batch_tune restore");
    }
    cudaFree(save_f);
    cudaFree(save_gray);
    cudaFree(save_macro);
    free_groups(b);
    free_graphs(b);
    if (rc != LBM_OK) return rc;
    b->tile_of_run = best;
    if (tiles_out)
        for (size_t r = 0; r < best.size(); ++r) tiles_out[r] = best[r];
    return LBM_OK;
}

int lbm_batch_info(lbm_batch *b, long long *cells, long long *steps, long long *launches, int *ngroups)
{
    if (!b) return LBM_ERR_ARG;
    if (cells) *cells = b->cells;
    if (steps) *steps = b->steps;
    if (launches) *launches = b->launches;
    if (ngroups) *ngroups = b->groups_ok ? (int)b->groups.size() : 0;
    return LBM_OK;
}

int lbm_batch_mss_to_saturation(lbm_batch *b, const double *targets, double gain, double max_rate, double tol,
                                int check_every, int max_steps, int *steps_done)
{
    if (!b || !targets || !steps_done || !(gain > 0.0) || !(max_rate > 0.0) || !(tol > 0.0) || check_every < 1 ||
        max_steps < 1 || !std::isfinite(gain) || !std::isfinite(max_rate))
        return LBM_ERR_ARG;
    const size_t nr = b->views.size();
    for (size_t r = 0; r < nr; ++r)
        if (!(targets[r] >= 0.0 && targets[r] <= 1.0)) return LBM_ERR_ARG;
    std::vector<lbm_obs> obs(nr);
    int done = 0, rc = LBM_OK;
    bool reached = false;
    while (rc == LBM_OK) {
        rc = lbm_batch_observables(b, obs.data());
        if (rc == LBM_ERR_NUMERIC) rc = LBM_OK;  // runs with non-finite fields are left out below
        if (rc != LBM_OK) break;
        reached = true;
        for (size_t r = 0; r < nr; ++r)
            reached = reached && (obs[r].nan_count > 0 || std::fabs(targets[r] - obs[r].sat) <= tol);
        if (reached || done >= max_steps) break;
        for (size_t r = 0; r < nr && rc == LBM_OK; ++r) {
            const double err = targets[r] - obs[r].sat;
            const double rate = (obs[r].nan_count > 0 || std::fabs(err) <= tol)
                                    ? 0.0
                                    : std::max(-max_rate, std::min(max_rate, gain * err));
            rc = lbm_set_mss(b->views[r], rate);
        }
        const int m = std::min(check_every, max_steps - done);
        if (rc == LBM_OK) rc = lbm_batch_step(b, m);
        done += m;
    }
    for (auto *v : b->views) lbm_set_mss(v, 0.0);
    *steps_done = done;
    if (rc != LBM_OK) return rc;
    return reached ? LBM_OK : LBM_ERR_TIMEOUT;
}

int lbm_batch_step_to_steady(lbm_batch *b, int check_every, double rel_tol, int max_steps, int *steps_done)
{
    if (!b || check_every < 1 || !(rel_tol > 0.0) || max_steps < 0) return LBM_ERR_ARG;
    const size_t nr = b->views.size();
    std::vector<lbm_obs> prev(nr), cur(nr);
    int rc = lbm_batch_observables(b, prev.data());
    if (rc != LBM_OK && rc != LBM_ERR_NUMERIC) return rc;
    int done = 0;
    bool steady = false;
    while (!steady && done < max_steps) {
        const int k = std::min(check_every, max_steps - done);
        rc = lbm_batch_step(b, k);
        if (rc != LBM_OK) return rc;
        done += k;
        rc = lbm_batch_observables(b, cur.data());
        if (rc != LBM_OK && rc != LBM_ERR_NUMERIC) return rc;
        steady = true;
        for (size_t r = 0; r < nr && steady; ++r) {
            if (cur[r].nan_count > 0) continue;  // non-finite runs are left out (see lbm_batch_observables)
            for (int d = 0; d < 3; ++d) {
                const double a = cur[r].flux_vol[d], p = prev[r].flux_vol[d];
                const double scale = std::max({std::fabs(cur[r].flux_vol[0]), std::fabs(cur[r].flux_vol[1]),
                                               std::fabs(cur[r].flux_vol[2]), 1e-300});
                if (std::fabs(a - p) > rel_tol * scale) {
                    steady = false;
                    break;
                }
            }
        }
        prev.swap(cur);
    }
    if (steps_done) *steps_done = done;
    return steady ? LBM_OK : LBM_ERR_TIMEOUT;
}

int lbm_batch_observables(lbm_batch *b, lbm_obs *out)
{
    if (!b || !out) return LBM_ERR_ARG;
    int worst = LBM_OK;
    for (size_t r = 0; r < b->views.size(); ++r) {
        const int rc = lbm_observables(b->views[r], &out[r]);
        if (rc == LBM_ERR_NUMERIC) worst = LBM_ERR_NUMERIC;
        else if (rc != LBM_OK) return rc;
    }
    return worst;
}

}  // extern "C"

// A view changed a per-run parameter (reservoir densities, mass-sink-source
// rate): the item tables, which carry them, are uploaded again before the
// next step.
void lbm::batch_runs_changed(lbm_batch *b)
{
    if (b) b->runs_dirty = true;
}
