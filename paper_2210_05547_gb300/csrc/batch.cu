// Batched execution: the RK3 steps of many independent grids (different sizes, freestreams, time
// steps) in shared launches, for serving many solves on one GPU.
//
// A batch joins its members' launch plans. Every line phase is one k_lines launch over the
// concatenation of the members' jobs; every pointwise step is one persistent kernel whose blocks
// walk a list of tiles (fixed-size index ranges of one member each), so members of uneven size
// share the SMs without a launch per member. The kernels run the same device bodies as the
// single-grid path (pointwise.cuh, lines.cu) on each member's own scratch, plan and caches, so a
// member's results are bit-identical whether it runs alone (hyp_rk_stage) or in any batch.
// A step can be captured once into a CUDA graph and replayed while the membership is unchanged.
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "grid.h"
#include "internal.h"
#include "pointwise.cuh"

using namespace hyp;

namespace {

// index spaces of the pointwise steps
enum Space { SP_NC, SP_FACES, SP_NCN, SP_GAUSS, SP_STATE, SP_FILTER, SP_COUNT };

struct alignas(8) BatchItem {
    GridView v;
    Scratch s;
    Scales sc;
    const double* U;
    AssembleArgs asmb;           // A and B are set per stage by the launch
    double filter_sigma;
    int cneq;
    long long n[SP_COUNT];
};

struct BatchDev {
    BatchItem* items;
    int nitems;
    int tile;                    // points per tile
    const int* tstart[SP_COUNT]; // per space: cumulative tile counts, nitems + 1 entries
};

// Blocks walk the tiles of one index space; the member of a tile is found by scanning the
// cumulative tile counts forward (a batch holds tens of members).
// The item table is read through a __restrict__ kernel parameter so that the compiler keeps the
// member's field pointers in registers across the stores made through them.
template <typename F>
__device__ __forceinline__ void for_tiles(const BatchItem* __restrict__ items, const BatchDev& B,
                                          int space, F&& f) {
    const int* __restrict__ ts = B.tstart[space];
    const int total = ts[B.nitems];
    int k = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        while (ts[k + 1] <= t) ++k;
        const BatchItem& it = items[k];
        const long long lo = (long long)(t - ts[k]) * B.tile;
        const long long hi = min(lo + B.tile, it.n[space]);
        f(it, lo, hi);
    }
}

// The closure touches about sixty fields of its member: the block copies the member's item into
// shared memory when it moves to a tile of another member, and the body reads the field
// pointers from there (no aliasing with the global stores, no registers held across the point).
template <bool MIXED, bool LTE>
__global__ void __launch_bounds__(128, CLOSURE_MIN_BLOCKS) kb_closure(const __grid_constant__ GasDev g,
                                                     const BatchItem* __restrict__ items,
                                                  BatchDev B) {
    __shared__ BatchItem sh;
    const int* __restrict__ ts = B.tstart[SP_NC];
    const int total = ts[B.nitems];
    int k = 0, cur = -1;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        while (ts[k + 1] <= t) ++k;
        if (k != cur) {
            __syncthreads();
            const long long* src = reinterpret_cast<const long long*>(items + k);
            long long* dst = reinterpret_cast<long long*>(&sh);
            for (int w = threadIdx.x; w < (int)(sizeof(BatchItem) / 8); w += blockDim.x) dst[w] = src[w];
            __syncthreads();
            cur = k;
        }
        const long long lo = (long long)(t - ts[k]) * B.tile;
        const long long hi = min(lo + B.tile, sh.n[SP_NC]);
        closure_body<MIXED, LTE>(g, sh.sc, sh.v, sh.U, sh.s, lo, hi, blockDim.x);
    }
}

__global__ void kb_face_vel(const BatchItem* __restrict__ items, BatchDev B) {
    for_tiles(items, B, SP_FACES, [&](const BatchItem& it, long long lo, long long hi) {
        face_vel_body(it.v, it.U, it.s, lo, hi, blockDim.x);
    });
}

__global__ void kb_ad_prep(const BatchItem* __restrict__ items, BatchDev B) {
    for_tiles(items, B, SP_NC, [&](const BatchItem& it, long long lo, long long hi) {
        if (it.v.ad) ad_prep_body(it.s, lo, hi, blockDim.x);
    });
}

__global__ void kb_ad_raw(const BatchItem* __restrict__ items, BatchDev B) {
    for_tiles(items, B, SP_NC, [&](const BatchItem& it, long long lo, long long hi) {
        if (it.v.ad) ad_raw_body(it.cneq != 0, it.v, it.U, it.s, lo, hi, blockDim.x);
    });
}

template <bool MIXED>
__global__ void kb_gauss(const BatchItem* __restrict__ items, BatchDev B, int dir) {
    for_tiles(items, B, SP_GAUSS, [&](const BatchItem& it, long long lo, long long hi) {
        if (it.v.ad) gauss_body<MIXED>(it.v, it.s, dir, lo, hi, blockDim.x);
    });
}

__global__ void kb_ad_combine(const BatchItem* __restrict__ items, BatchDev B) {
    for_tiles(items, B, SP_NC, [&](const BatchItem& it, long long lo, long long hi) {
        if (it.v.ad) ad_combine_body(it.s, lo, hi, blockDim.x);
    });
}

__global__ void kb_stress_c(const BatchItem* __restrict__ items, BatchDev B) {
    for_tiles(items, B, SP_NC, [&](const BatchItem& it, long long lo, long long hi) {
        stress_c_body(it.s, lo, hi, blockDim.x);
    });
}

__global__ void kb_stress_cn(const BatchItem* __restrict__ items, BatchDev B) {
    for_tiles(items, B, SP_NCN, [&](const BatchItem& it, long long lo, long long hi) {
        stress_cn_body(it.s, lo, hi, blockDim.x);
    });
}

template <bool SMK>
__global__ void kb_flux(GasDev g, const BatchItem* __restrict__ items, BatchDev B) {
    for_tiles(items, B, SP_FACES, [&](const BatchItem& it, long long lo, long long hi) {
        flux_body<SMK>(g, it.sc, it.v, it.U, it.s, -1, lo, hi, blockDim.x);
    });
}

__global__ void kb_assemble(const BatchItem* __restrict__ items, BatchDev B, double A, double Bc) {
    for_tiles(items, B, SP_STATE, [&](const BatchItem& it, long long lo, long long hi) {
        AssembleArgs a = it.asmb;
        a.A = A;
        a.B = Bc;
        assemble_body(a, lo, hi, blockDim.x);
    });
}

// x pass from the state into the member's state-sized scratch, y pass back (members with a
// filter only: the others have no tiles in SP_FILTER)
__global__ void kb_filter(const BatchItem* __restrict__ items, BatchDev B, int dir) {
    for_tiles(items, B, SP_FILTER, [&](const BatchItem& it, long long lo, long long hi) {
        double* U = it.asmb.U;
        const double* in = dir == 0 ? U : it.s.R;
        double* out = dir == 0 ? it.s.R : U;
        filter_body(it.v.nx, it.v.ny, in, out, dir, it.filter_sigma, lo, hi, blockDim.x);
    });
}

__global__ void kb_set_predict(BatchItem* items, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) items[k].v.predict = 1;
}

int device_sms() {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

struct hyp_batch {
    int precision = HYP_FP64;
    int tile = 512;
    int tile_auto = 1;           // pick the tile size by timing real steps after each change
    int tuned = 0;               // the tile size has been chosen for the current membership
    std::map<int, int> tile_cache;   // chosen tile per batch size class (log2 of the cell count)
    int use_graph = 0;
    GasDev table;                // gas tables shared by the members (freestream scales per member)
    bool have_table = false;
    struct Member {
        hyp_state* st;
        double dt;
    };
    std::vector<Member> members;
    bool dirty = true;
    // host images of the device tables (kept while their uploads may be in flight)
    std::vector<BatchItem> h_items;
    std::vector<int> h_tstart;
    std::vector<LineJob> h_jobs;
    BatchItem* d_items = nullptr;
    int* d_tstart = nullptr;
    LineJob* d_jobs = nullptr;
    size_t cap_items = 0, cap_jobs = 0;
    int ph_start[PH_COUNT] = {}, ph_count[PH_COUNT] = {}, ph_blocks[PH_COUNT] = {};
    int tiles[SP_COUNT] = {};
    int closure_blocks[4] = {0, 0, 0, 0};   // [mixed + 2 lte]: resident blocks of kb_closure
    bool any_sm = false;         // a member uses Stefan-Maxwell diffusion
    int pw_blocks = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t fork[2] = {}, join[2] = {};
    cudaGraphExec_t exec = nullptr;
    cudaStream_t gstream = nullptr;      // captures and replays the graph (any caller stream)
    cudaEvent_t g_in = nullptr, g_out = nullptr;
};

namespace {

void drop_graph(hyp_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

bool same_table(const GasDev& a, const GasDev& b) {
    return memcmp(&a, &b, offsetof(GasDev, rho_inf)) == 0;
}

BatchDev dev_view(const hyp_batch* b) {
    BatchDev B;
    B.items = b->d_items;
    B.nitems = (int)b->members.size();
    B.tile = b->tile;
    for (int sp = 0; sp < SP_COUNT; ++sp) B.tstart[sp] = b->d_tstart + (size_t)sp * (B.nitems + 1);
    return B;
}

// Rebuild the device item table, tile lists and the joined launch plan.
int rebuild(hyp_batch* b, cudaStream_t s) {
    const int n = (int)b->members.size();
    b->h_items.assign(n, BatchItem());
    b->h_tstart.assign((size_t)SP_COUNT * (n + 1), 0);
    b->h_jobs.clear();
    b->any_sm = false;
    for (int k = 0; k < n; ++k) {
        hyp_grid* G = b->members[k].st->grid;
        BatchItem& it = b->h_items[k];
        memset(&it, 0, sizeof(it));
        it.v = G->view();
        b->any_sm = b->any_sm || it.v.sm;
        it.s = G->s;
        it.sc = scales_of(G->gas);
        it.U = b->members[k].st->U;
        it.asmb = AssembleArgs{G->s.DX, G->s.DY, G->s.SRC, G->sigma, G->Uref, G->mask,
                               b->members[k].st->U, nullptr, b->members[k].st->dQ, 1, 0.0, 0.0,
                               b->members[k].dt};
        it.filter_sigma = G->cas.filter_sigma;
        it.cneq = G->gas.kind == HYP_GAS_CNEQ;
        const long long nc = G->d.size(hyp::NC);
        it.n[SP_NC] = nc;
        it.n[SP_FACES] = G->d.size(hyp::NXF) + G->d.size(hyp::NYF);
        it.n[SP_NCN] = G->d.size(hyp::NCN);
        // the binary32 filter's threads take every field of a point (gauss_body)
        it.n[SP_GAUSS] = b->precision == HYP_MIXED ? nc : (long long)AD_FIELDS * nc;
        it.n[SP_STATE] = G->nstate;
        it.n[SP_FILTER] = G->cas.filter_sigma > 0.0 ? G->nstate : 0;
    }
    for (int sp = 0; sp < SP_COUNT; ++sp) {
        int* ts = b->h_tstart.data() + (size_t)sp * (n + 1);
        for (int k = 0; k < n; ++k)
            ts[k + 1] = ts[k] + (int)((b->h_items[k].n[sp] + b->tile - 1) / b->tile);
        b->tiles[sp] = ts[n];
    }
    for (int ph = 0; ph < PH_COUNT; ++ph) {
        b->ph_start[ph] = (int)b->h_jobs.size();
        b->ph_blocks[ph] = 0;
        for (int k = 0; k < n; ++k) {
            hyp_grid* G = b->members[k].st->grid;
            if ((ph == PH_AD1 || ph == PH_AD2) && !G->cas.artificial_diffusivity) continue;
            for (int q = 0; q < G->ph_count[ph]; ++q) {
                LineJob j = G->hjobs[G->ph_start[ph] + q];
                if (j.in_state) {
                    j.in = b->members[k].st->U + (size_t)j.in;
                    j.in_state = 0;
                }
                b->h_jobs.push_back(j);
            }
            b->ph_blocks[ph] = std::max(b->ph_blocks[ph], G->ph_blocks[ph]);
        }
        b->ph_count[ph] = (int)b->h_jobs.size() - b->ph_start[ph];
    }
    cudaError_t e = cudaSuccess;
    if ((size_t)n > b->cap_items) {
        cudaFree(b->d_items);
        cudaFree(b->d_tstart);
        b->d_items = nullptr;
        b->d_tstart = nullptr;
        b->cap_items = 0;
        const size_t cap = std::max<size_t>(16, 2 * n);
        e = cudaMalloc(&b->d_items, cap * sizeof(BatchItem));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_tstart, (size_t)SP_COUNT * (cap + 1) * sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(batch items)");
        b->cap_items = cap;
    }
    if (b->h_jobs.size() > b->cap_jobs) {
        cudaFree(b->d_jobs);
        b->d_jobs = nullptr;
        b->cap_jobs = 0;
        const size_t cap = std::max<size_t>(256, 2 * b->h_jobs.size());
        e = cudaMalloc(&b->d_jobs, cap * sizeof(LineJob));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(batch jobs)");
        b->cap_jobs = cap;
    }
    if (n) {
        HYP_CUDA(cudaMemcpyAsync(b->d_items, b->h_items.data(), n * sizeof(BatchItem),
                                 cudaMemcpyHostToDevice, s));
        HYP_CUDA(cudaMemcpyAsync(b->d_tstart, b->h_tstart.data(), b->h_tstart.size() * sizeof(int),
                                 cudaMemcpyHostToDevice, s));
    }
    if (!b->h_jobs.empty())
        HYP_CUDA(cudaMemcpyAsync(b->d_jobs, b->h_jobs.data(), b->h_jobs.size() * sizeof(LineJob),
                                 cudaMemcpyHostToDevice, s));
    HYP_CUDA(cudaStreamSynchronize(s));   // the host images may change on the next rebuild
    b->dirty = false;
    drop_graph(b);
    return HYP_OK;
}

int grid_for_tiles(const hyp_batch* b, int space, int cap) {
    return std::max(1, std::min(b->tiles[space], cap));
}

// One RK3 step (three stages and the state filter) of every member, enqueued on s.
int launch_step(hyp_batch* b, cudaStream_t s) {
    const BatchDev B = dev_view(b);
    const int mixed = b->precision == HYP_MIXED ? 1 : 0;
    const int pw = b->pw_blocks;
    cudaStream_t s2 = b->side;
    // the sensors' cross-derivative interpolations (PH_AD1, PH_AD2) run in binary64 in both
    // precisions, as in run_rhs
    auto lines = [&](int ph, cudaStream_t st) {
        const int mx = (ph == PH_AD1 || ph == PH_AD2) ? 0 : mixed;
        return launch_lines(b->d_jobs + b->ph_start[ph], b->ph_count[ph], b->ph_blocks[ph],
                            nullptr, st, mx);
    };
    for (int stage = 0; stage < 3; ++stage) {
        HYP_CUDA(lines(PH_P1, s));
        kb_face_vel<<<grid_for_tiles(b, SP_FACES, pw), 256, 0, s>>>(b->d_items, B);
        HYP_CUDA(cudaEventRecord(b->fork[0], s));
        HYP_CUDA(cudaStreamWaitEvent(s2, b->fork[0], 0));
        const int cb = grid_for_tiles(
            b, SP_NC, b->closure_blocks[mixed + (b->table.kind == HYP_GAS_LTE ? 2 : 0)]);
        if (b->table.kind == HYP_GAS_LTE) {
            if (mixed) kb_closure<true, true><<<cb, 128, 0, s>>>(b->table, b->d_items, B);
            else kb_closure<false, true><<<cb, 128, 0, s>>>(b->table, b->d_items, B);
        } else {
            if (mixed) kb_closure<true, false><<<cb, 128, 0, s>>>(b->table, b->d_items, B);
            else kb_closure<false, false><<<cb, 128, 0, s>>>(b->table, b->d_items, B);
        }
        kb_set_predict<<<(B.nitems + 127) / 128, 128, 0, s>>>(b->d_items, B.nitems);
        HYP_CUDA(lines(PH_P3, s2));
        HYP_CUDA(lines(PH_AD1, s2));
        HYP_CUDA(lines(PH_AD2, s2));
        kb_ad_prep<<<grid_for_tiles(b, SP_NC, pw), 256, 0, s2>>>(b->d_items, B);
        HYP_CUDA(cudaEventRecord(b->join[0], s2));
        HYP_CUDA(cudaStreamWaitEvent(s, b->join[0], 0));
        kb_ad_raw<<<grid_for_tiles(b, SP_NC, pw), 256, 0, s>>>(b->d_items, B);
        if (mixed) {
            kb_gauss<true><<<grid_for_tiles(b, SP_GAUSS, pw), 256, 0, s>>>(b->d_items, B, 0);
            kb_gauss<true><<<grid_for_tiles(b, SP_GAUSS, pw), 256, 0, s>>>(b->d_items, B, 1);
        } else {
            kb_gauss<false><<<grid_for_tiles(b, SP_GAUSS, pw), 256, 0, s>>>(b->d_items, B, 0);
            kb_gauss<false><<<grid_for_tiles(b, SP_GAUSS, pw), 256, 0, s>>>(b->d_items, B, 1);
        }
        kb_ad_combine<<<grid_for_tiles(b, SP_NC, pw), 256, 0, s>>>(b->d_items, B);
        kb_stress_c<<<grid_for_tiles(b, SP_NC, pw), 256, 0, s>>>(b->d_items, B);
        HYP_CUDA(cudaGetLastError());
        HYP_CUDA(cudaEventRecord(b->fork[1], s));
        HYP_CUDA(cudaStreamWaitEvent(s2, b->fork[1], 0));
        HYP_CUDA(lines(PH_MU1, s2));
        HYP_CUDA(lines(PH_MU2, s2));
        kb_stress_cn<<<grid_for_tiles(b, SP_NCN, pw), 256, 0, s2>>>(b->d_items, B);
        HYP_CUDA(lines(PH_FACEB, s2));
        HYP_CUDA(cudaEventRecord(b->join[1], s2));
        HYP_CUDA(lines(PH_FACE, s));
        HYP_CUDA(cudaStreamWaitEvent(s, b->join[1], 0));
        if (b->any_sm) kb_flux<true><<<grid_for_tiles(b, SP_FACES, pw), 128, 0, s>>>(b->table, b->d_items, B);
        else kb_flux<false><<<grid_for_tiles(b, SP_FACES, pw), 128, 0, s>>>(b->table, b->d_items, B);
        HYP_CUDA(lines(PH_DIV, s));
        kb_assemble<<<grid_for_tiles(b, SP_STATE, pw), 256, 0, s>>>(b->d_items, B, RK_A[stage], RK_B[stage]);
        HYP_CUDA(cudaGetLastError());
    }
    if (b->tiles[SP_FILTER]) {
        kb_filter<<<grid_for_tiles(b, SP_FILTER, pw), 256, 0, s>>>(b->d_items, B, 0);
        kb_filter<<<grid_for_tiles(b, SP_FILTER, pw), 256, 0, s>>>(b->d_items, B, 1);
        HYP_CUDA(cudaGetLastError());
    }
    return HYP_OK;
}

}  // namespace

extern "C" int hyp_batch_create(int precision, hyp_batch** out) {
    if (!out) return fail(HYP_ERR_ARG, "null output");
    if (precision != HYP_FP64 && precision != HYP_MIXED) return fail(HYP_ERR_ARG, "unknown precision");
    hyp_batch* b = new hyp_batch();
    b->precision = precision;
    cudaError_t e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->g_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->g_out, cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&b->fork[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
    }
    int per_sm = 0;
    const int sms = device_sms();
    {
        void (*const kern[4])(GasDev, const BatchItem*, BatchDev) = {
            kb_closure<false, false>, kb_closure<true, false>, kb_closure<false, true>,
            kb_closure<true, true>};
        for (int q = 0; q < 4; ++q) {
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern[q], 128, 0);
            b->closure_blocks[q] = std::max(1, per_sm * sms);
        }
    }
    b->pw_blocks = sms * 8;
    if (e != cudaSuccess) {
        hyp_batch_free(b);
        return cuda_fail(e, "batch set-up");
    }
    *out = b;
    return HYP_OK;
}

extern "C" int hyp_batch_add(hyp_batch* b, hyp_state* st, double dt) {
    if (!b || !st) return fail(HYP_ERR_ARG, "null argument");
    if (!(dt >= 0.0)) return fail(HYP_ERR_ARG, "time step must be >= 0");
    if (st->grid->g3) return fail(HYP_ERR_ARG, "the batch takes two-dimensional grids");
    for (const auto& m : b->members)
        if (m.st == st) return fail(HYP_ERR_ARG, "state is already in the batch");
    const GasDev& g = st->grid->gas;
    if (!b->have_table) {
        b->table = g;
        b->have_table = true;
    } else if (!same_table(b->table, g)) {
        return fail(HYP_ERR_ARG, "batch members must share one gas table and kind");
    }
    b->members.push_back({st, dt});
    b->dirty = true;
    b->tuned = 0;
    return HYP_OK;
}

extern "C" int hyp_batch_remove(hyp_batch* b, hyp_state* st) {
    if (!b || !st) return fail(HYP_ERR_ARG, "null argument");
    for (size_t k = 0; k < b->members.size(); ++k) {
        if (b->members[k].st == st) {
            b->members.erase(b->members.begin() + k);
            b->dirty = true;
            b->tuned = 0;
            if (b->members.empty()) b->have_table = false;
            return HYP_OK;
        }
    }
    return fail(HYP_ERR_ARG, "state is not in the batch");
}

extern "C" int hyp_batch_configure(hyp_batch* b, int use_graph, int tile) {
    if (!b) return fail(HYP_ERR_ARG, "null batch");
    if (tile < 0 || (tile > 0 && tile % 128 != 0)) return fail(HYP_ERR_ARG, "tile must be a positive multiple of 128");
    if (tile > 0 && tile != b->tile) {
        b->tile = tile;
        b->dirty = true;
    }
    b->tile_auto = tile == 0;
    if ((use_graph != 0) != (b->use_graph != 0)) drop_graph(b);
    b->use_graph = use_graph != 0;
    return HYP_OK;
}

extern "C" int hyp_batch_size(const hyp_batch* b, int* members) {
    if (!b || !members) return fail(HYP_ERR_ARG, "null argument");
    *members = (int)b->members.size();
    return HYP_OK;
}

extern "C" int hyp_batch_tile(const hyp_batch* b, int* tile, int* tuned) {
    if (!b) return fail(HYP_ERR_ARG, "null batch");
    if (tile) *tile = b->tile;
    if (tuned) *tuned = b->tile_auto ? b->tuned : 1;
    return HYP_OK;
}

extern "C" int hyp_batch_step(hyp_batch* b, int nsteps, void* stream) {
    if (!b || nsteps < 0) return fail(HYP_ERR_ARG, "null batch or negative step count");
    if (b->members.empty() || nsteps == 0) return HYP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (b->dirty) {
        const int rc = rebuild(b, s);
        if (rc) return rc;
    }
    for (auto& m : b->members) m.st->grid->cache_valid = 1;   // after this call's first closure
    // Autotuner: the tile size only distributes work (every point is computed the same way), so
    // candidate tiles are timed on real steps of the solution: one untimed step after a change
    // of membership, then one timed step per candidate, then the fastest is kept.
    long long cells = 0;
    for (const auto& m : b->members) cells += m.st->grid->d.size(hyp::NC);
    int size_class = 0;
    while ((2LL << size_class) <= cells) ++size_class;
    if (b->tile_auto && !b->tuned) {
        auto hit = b->tile_cache.find(size_class);
        if (hit != b->tile_cache.end()) {
            b->tuned = 1;
            if (b->tile != hit->second) {
                b->tile = hit->second;
                const int rc = rebuild(b, s);
                if (rc) return rc;
            }
        }
    }
    if (b->tile_auto && !b->tuned) {
        static const int cand[] = {256, 512, 1024, 2048};
        float best_ms = 0.0f;
        int best = b->tile;
        cudaEvent_t e0, e1;
        HYP_CUDA(cudaEventCreate(&e0));
        HYP_CUDA(cudaEventCreate(&e1));
        int rc = HYP_OK;
        if (nsteps > 0) {
            rc = launch_step(b, s);
            --nsteps;
        }
        for (int c = 0; c < 4 && nsteps > 0 && rc == HYP_OK; ++c) {
            b->tile = cand[c];
            if ((rc = rebuild(b, s))) break;
            cudaEventRecord(e0, s);
            if ((rc = launch_step(b, s))) break;
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (c == 0 || ms < best_ms) {
                best_ms = ms;
                best = cand[c];
            }
            --nsteps;
            if (c == 3) {
                b->tuned = 1;
                b->tile_cache[size_class] = best;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) return rc;
        if (b->tile != best) {
            b->tile = best;
            if ((rc = rebuild(b, s))) return rc;
        }
        if (nsteps == 0) return HYP_OK;
    }
    if (!b->use_graph) {
        for (int k = 0; k < nsteps; ++k) {
            const int rc = launch_step(b, s);
            if (rc) return rc;
        }
        return HYP_OK;
    }
    // the graph is captured on and replayed from the batch's own stream (capture is not possible
    // on the legacy default stream), ordered after and before the caller's stream by events
    if (!b->exec) {
        cudaGraph_t graph = nullptr;
        HYP_CUDA(cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal));
        const int rc = launch_step(b, b->gstream);
        const cudaError_t ec = cudaStreamEndCapture(b->gstream, &graph);
        if (rc || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return rc ? rc : cuda_fail(ec, "cudaStreamEndCapture");
        }
        const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            b->exec = nullptr;
            cudaGetLastError();
            return cuda_fail(ei, "cudaGraphInstantiate");
        }
    }
    HYP_CUDA(cudaEventRecord(b->g_in, s));
    HYP_CUDA(cudaStreamWaitEvent(b->gstream, b->g_in, 0));
    for (int k = 0; k < nsteps; ++k) HYP_CUDA(cudaGraphLaunch(b->exec, b->gstream));
    HYP_CUDA(cudaEventRecord(b->g_out, b->gstream));
    HYP_CUDA(cudaStreamWaitEvent(s, b->g_out, 0));
    return HYP_OK;
}

extern "C" void hyp_batch_free(hyp_batch* b) {
    if (!b) return;
    drop_graph(b);
    cudaFree(b->d_items);
    cudaFree(b->d_tstart);
    cudaFree(b->d_jobs);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->gstream) cudaStreamDestroy(b->gstream);
    if (b->g_in) cudaEventDestroy(b->g_in);
    if (b->g_out) cudaEventDestroy(b->g_out);
    for (int k = 0; k < 2; ++k) {
        if (b->fork[k]) cudaEventDestroy(b->fork[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    delete b;
}
