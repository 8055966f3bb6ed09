// Ragged batches: arrays of mixed shapes transformed by one graph launch.
//
// The paper's interface transforms one array per call and loops in C
// (Section 3.2); on the GPU a batch of mixed shapes is grouped into shape
// classes, each served by the fastest accepted path for its shape, and every
// class is one persistent kernel launch that reads its arrays through a
// device table of element offsets.  The launches of all classes are captured
// once into a CUDA graph per (direction, base pointers) and replayed.
//
// Path choice per class (the paper fixes its policy per size before
// measuring, Section 3.2; here it is measured): the accepted candidates (the
// FP32 route for the shape, and the split-BF16 tensor-core route where it
// exists) are timed on scratch arrays of the class's shape when the ragged
// plan is created; report-only paths never compete.  With BDCT_TUNE_CACHE set
// to a file path, choices are read from and appended to that file (one line
// "rows cols kind norm path us_per_array").
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "bdct_internal.h"
#include "plan.h"

using namespace bdct;

namespace {

struct RaggedClass {
    int rows = 0, cols = 0;
    std::vector<long long> in_off, out_off;  // element offsets (host copy)
    long long *d_in_off = nullptr, *d_out_off = nullptr;
    long long elems = 0;  // total elements of the class
    bdct_plan *plan = nullptr;
    int path = 0;
    size_t chunk_bytes = 0;  // separable routes: workspace chunk chosen (0 = none)
    double tuned_us = 0.0;  // measured time per array of the chosen path (0 = not measured)
};

struct GraphEntry {
    unsigned kind;
    const float *in;
    float *out;
    cudaGraphExec_t exec;
};

std::mutex g_cache_mutex;

const char *tune_cache_path() { return getenv("BDCT_TUNE_CACHE"); }

bool cache_lookup(int rows, int cols, unsigned kind, int norm, int *path, size_t *chunk_mb)
{
    const char *fn = tune_cache_path();
    if (!fn) return false;
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    FILE *f = fopen(fn, "r");
    if (!f) return false;
    int r, c, n, pth;
    unsigned k;
    size_t mb;
    double us;
    bool found = false;
    while (fscanf(f, "%d %d %u %d %d %zu %lf", &r, &c, &k, &n, &pth, &mb, &us) == 7) {
        if (r == rows && c == cols && k == kind && n == norm &&
            (pth == BDCT_PATH_FP32 || pth == BDCT_PATH_SPLIT_TC)) {
            *path = pth;  // the last entry wins
            *chunk_mb = mb;
            found = true;
        }
    }
    fclose(f);
    return found;
}

void cache_store(int rows, int cols, unsigned kind, int norm, int path, size_t chunk_mb, double us)
{
    const char *fn = tune_cache_path();
    if (!fn) return;
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    FILE *f = fopen(fn, "a");
    if (!f) return;
    fprintf(f, "%d %d %u %d %d %zu %.4f\n", rows, cols, kind, norm, path, chunk_mb, us);
    fclose(f);
}

}  // namespace

struct bdct_ragged {
    int device = -1;
    unsigned kind = 0;
    int norm = 0;
    std::vector<RaggedClass> classes;  // largest first
    cudaStream_t capture = nullptr;
    std::mutex mu;
    std::vector<GraphEntry> graphs;
};

static void ragged_free(bdct_ragged *r)
{
    if (!r) return;
    for (auto &g : r->graphs) cudaGraphExecDestroy(g.exec);
    for (auto &c : r->classes) {
        if (c.d_in_off) cudaFree(c.d_in_off);
        if (c.d_out_off) cudaFree(c.d_out_off);
        if (c.plan) bdct_plan_destroy(c.plan);
    }
    if (r->capture) cudaStreamDestroy(r->capture);
    delete r;
}

// Time `reps` forward calls of `plan` on `n` scratch arrays; microseconds per array.
static int time_plan(bdct_plan *plan, unsigned kind_mask, float *d_in, float *d_out, long long n, double *us)
{
    // warm every planned direction once (also sets up each kernel before any capture)
    const unsigned kinds[3] = {BDCT_FORWARD, BDCT_INVERSE, BDCT_ROUNDTRIP};
    for (unsigned k : kinds)
        if (kind_mask & k) {
            int st = bdct_execute(plan, k, d_in, d_out, (size_t)n, nullptr);
            if (st != BDCT_OK) return st;
        }
    if (cudaDeviceSynchronize() != cudaSuccess) return BDCT_ERR_CUDA;
    const unsigned tk = (kind_mask & BDCT_FORWARD) ? BDCT_FORWARD : ((kind_mask & BDCT_INVERSE) ? BDCT_INVERSE : BDCT_ROUNDTRIP);
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return BDCT_ERR_CUDA;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return BDCT_ERR_CUDA; }
    const int reps = 5;
    cudaEventRecord(a, nullptr);
    int st = BDCT_OK;
    for (int i = 0; i < reps && st == BDCT_OK; ++i) st = bdct_execute(plan, tk, d_in, d_out, (size_t)n, nullptr);
    cudaEventRecord(b, nullptr);
    float ms = 0.f;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) st = BDCT_ERR_CUDA;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *us = (double)ms * 1e3 / reps / (double)n;
    return st;
}

// Pick and create the plan of one class: the accepted candidate paths (FP32,
// and the on-chip split-BF16 tensor-core route where it exists), and for a
// separable route the workspace chunk (64, 128 or 256 MiB: every chunk
// costs two launches with their ramp-up and drain, which measured more than
// keeping the intermediate in L2 -- 256^2 batches ran at 0.19 / 0.31 / 0.34
// of HBM with 8 / 64 / 128 MiB chunks), each timed on scratch arrays of the
// class's shape.
static int class_plan(RaggedClass &c, unsigned kind, int norm, int path)
{
    const bool tc_ok = tc_supported(c.rows, c.cols);
    if (path != BDCT_PATH_AUTO) {
        c.path = path;
        return bdct_plan_create(&c.plan, c.rows, c.cols, kind, norm, path);
    }
    const long long arr = (long long)c.rows * c.cols;
    const bool separable = !fused_supported(c.rows, c.cols);
    // scratch: 32 MiB, or 512 MiB where chunk sizes are compared
    long long n = ((separable ? 512ll : 32ll) << 20) / (arr * 4);
    if (n < 1) n = 1;
    if (n > (long long)c.in_off.size()) n = (long long)c.in_off.size();
    float *d_in = nullptr, *d_out = nullptr;
    if (cudaMalloc(&d_in, (size_t)n * arr * 4) != cudaSuccess) return BDCT_ERR_NO_MEMORY;
    if (cudaMalloc(&d_out, (size_t)n * arr * 4) != cudaSuccess) { cudaFree(d_in); return BDCT_ERR_NO_MEMORY; }
    cudaMemset(d_in, 0, (size_t)n * arr * 4);

    struct Cand { int path; size_t chunk_mb; };
    std::vector<Cand> cands;
    int cached = 0;
    size_t cached_mb = 0;
    if (cache_lookup(c.rows, c.cols, kind, norm, &cached, &cached_mb)) {
        cands.push_back({cached, cached_mb});
    } else if (separable) {
        for (size_t mb : {64, 128, 256}) cands.push_back({BDCT_PATH_FP32, mb});
    } else {
        cands.push_back({BDCT_PATH_FP32, 0});
        if (tc_ok) cands.push_back({BDCT_PATH_SPLIT_TC, 0});
    }
    int st = BDCT_OK;
    double best = 1e300;
    bdct_plan *pl = nullptr;
    int pl_path = -1;
    for (const Cand &cd : cands) {
        if (cd.path != pl_path) {
            if (pl && pl != c.plan) bdct_plan_destroy(pl);
            pl = nullptr;
            st = bdct_plan_create(&pl, c.rows, c.cols, kind, norm, cd.path);
            if (st != BDCT_OK) break;
            pl_path = cd.path;
        }
        if (cd.chunk_mb) {
            st = bdct_plan_set_chunk_bytes(pl, cd.chunk_mb << 20);
            if (st != BDCT_OK) break;
        }
        double us = 0.0;
        st = time_plan(pl, kind, d_in, d_out, n, &us);
        if (st != BDCT_OK) break;
        if (us < best) {
            best = us;
            c.path = cd.path;
            c.chunk_bytes = cd.chunk_mb << 20;
            if (c.plan && c.plan != pl) bdct_plan_destroy(c.plan);
            c.plan = pl;
        }
    }
    if (pl && pl != c.plan) bdct_plan_destroy(pl);
    cudaFree(d_in);
    cudaFree(d_out);
    if (st != BDCT_OK) return st;
    // the same plan may have been timed at a later chunk size than the best one
    if (c.chunk_bytes) {
        st = bdct_plan_set_chunk_bytes(c.plan, c.chunk_bytes);
        if (st != BDCT_OK) return st;
    }
    c.tuned_us = best;
    if (cands.size() > 1) cache_store(c.rows, c.cols, kind, norm, c.path, c.chunk_bytes >> 20, best);
    return BDCT_OK;
}

extern "C" int bdct_ragged_create(bdct_ragged **out, size_t n, const int *rows, const int *cols, const size_t *in_off,
                                  const size_t *out_off, unsigned kind, int norm, int path)
{
    if (!out) return BDCT_ERR_INVALID_ARG;
    *out = nullptr;
    if ((n > 0 && (!rows || !cols || !in_off || !out_off)) || kind == 0 ||
        (kind & ~(BDCT_FORWARD | BDCT_INVERSE | BDCT_ROUNDTRIP)))
        return BDCT_ERR_INVALID_ARG;
    if (norm != BDCT_NORM_ORTHO && norm != BDCT_NORM_NONE) return BDCT_ERR_INVALID_ARG;
    if (path != BDCT_PATH_AUTO && path != BDCT_PATH_FP32 && path != BDCT_PATH_SPLIT_TC) return BDCT_ERR_PATH;
    for (size_t i = 0; i < n; ++i) {
        if (rows[i] < 1 || cols[i] < 1) return BDCT_ERR_INVALID_ARG;
        if (rows[i] > 8192 || cols[i] > 8192 || cols[i] % 4) return BDCT_ERR_UNSUPPORTED_SHAPE;
        if ((in_off[i] | out_off[i]) & 3u) return BDCT_ERR_ALIGN;
    }
    bdct_ragged *r = new (std::nothrow) bdct_ragged;
    if (!r) return BDCT_ERR_NO_MEMORY;
    if (cudaGetDevice(&r->device) != cudaSuccess) { delete r; return BDCT_ERR_CUDA; }
    r->kind = kind;
    r->norm = norm;
    // group by shape
    std::map<std::pair<int, int>, size_t> idx;
    for (size_t i = 0; i < n; ++i) {
        const auto key = std::make_pair(rows[i], cols[i]);
        auto it = idx.find(key);
        if (it == idx.end()) {
            it = idx.emplace(key, r->classes.size()).first;
            RaggedClass c;
            c.rows = rows[i];
            c.cols = cols[i];
            r->classes.push_back(std::move(c));
        }
        RaggedClass &c = r->classes[it->second];
        c.in_off.push_back((long long)in_off[i]);
        c.out_off.push_back((long long)out_off[i]);
        c.elems += (long long)rows[i] * cols[i];
    }
    std::sort(r->classes.begin(), r->classes.end(),
              [](const RaggedClass &a, const RaggedClass &b) { return a.elems > b.elems; });
    for (auto &c : r->classes) {
        int st = class_plan(c, kind, norm, path);
        if (st != BDCT_OK) { ragged_free(r); return st; }
        const size_t bytes = c.in_off.size() * sizeof(long long);
        if (cudaMalloc(&c.d_in_off, bytes) != cudaSuccess || cudaMalloc(&c.d_out_off, bytes) != cudaSuccess) {
            ragged_free(r);
            return BDCT_ERR_NO_MEMORY;
        }
        if (cudaMemcpy(c.d_in_off, c.in_off.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c.d_out_off, c.out_off.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            ragged_free(r);
            return BDCT_ERR_CUDA;
        }
    }
    if (cudaStreamCreateWithFlags(&r->capture, cudaStreamNonBlocking) != cudaSuccess) {
        ragged_free(r);
        return BDCT_ERR_CUDA;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) { ragged_free(r); return BDCT_ERR_CUDA; }
    *out = r;
    return BDCT_OK;
}

// Record every class's launch, largest class first, into the capture
// stream's graph.  (Parallel graph branches per class, on side streams forked
// from the capture stream, measured slower on the 4096-array workload: 0.217
// to 0.229 of HBM against 0.241 serial -- every class kernel is persistent
// and sized to fill the GPU, so branches only contend.)
static int ragged_launch_all(const bdct_ragged *r, Dir dir, const float *in, float *out)
{
    for (const auto &c : r->classes) {
        const int st = plan_execute(c.plan, dir, in, c.d_in_off, out, c.d_out_off, (long long)c.in_off.size(),
                                    r->capture);
        if (st != BDCT_OK) return st;
    }
    return BDCT_OK;
}

extern "C" int bdct_ragged_execute(bdct_ragged *r, unsigned kind, const float *in_base, float *out_base,
                                   void *stream)
{
    if (!r) return BDCT_ERR_INVALID_ARG;
    Dir dir;
    switch (kind) {
        case BDCT_FORWARD: dir = DIR_FWD; break;
        case BDCT_INVERSE: dir = DIR_INV; break;
        case BDCT_ROUNDTRIP: dir = DIR_RT; break;
        default: return BDCT_ERR_INVALID_ARG;
    }
    if (!(r->kind & kind)) return BDCT_ERR_KIND;
    if (r->classes.empty()) return BDCT_OK;
    if (!in_base || !out_base) return BDCT_ERR_INVALID_ARG;
    if (((uintptr_t)in_base | (uintptr_t)out_base) & 15u) return BDCT_ERR_ALIGN;
    std::lock_guard<std::mutex> lock(r->mu);
    cudaGraphExec_t exec = nullptr;
    for (const auto &g : r->graphs)
        if (g.kind == kind && g.in == in_base && g.out == out_base) exec = g.exec;
    if (!exec) {
        // capture every class's launch once for these pointers
        if (cudaStreamBeginCapture(r->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BDCT_ERR_CUDA;
        int st = ragged_launch_all(r, dir, in_base, out_base);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(r->capture, &graph);
        if (st != BDCT_OK) { if (graph) cudaGraphDestroy(graph); return st; }
        if (e != cudaSuccess) return BDCT_ERR_CUDA;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return BDCT_ERR_CUDA;
        r->graphs.push_back(GraphEntry{kind, in_base, out_base, exec});
    }
    if (cudaGraphLaunch(exec, (cudaStream_t)stream) != cudaSuccess) return BDCT_ERR_CUDA;
    return BDCT_OK;
}

extern "C" int bdct_ragged_destroy(bdct_ragged *r)
{
    if (!r) return BDCT_OK;
    ragged_free(r);
    return BDCT_OK;
}

extern "C" int bdct_ragged_num_classes(const bdct_ragged *r)
{
    if (!r) return -BDCT_ERR_INVALID_ARG;
    return (int)r->classes.size();
}

extern "C" int bdct_ragged_class_info(const bdct_ragged *r, int index, bdct_ragged_class *info)
{
    if (!r || !info || index < 0 || index >= (int)r->classes.size()) return BDCT_ERR_INVALID_ARG;
    const RaggedClass &c = r->classes[(size_t)index];
    info->rows = c.rows;
    info->cols = c.cols;
    info->count = c.in_off.size();
    info->path = c.path == BDCT_PATH_AUTO ? c.plan->path : c.path;
    info->variant = c.plan->variant;
    info->tuned_us_per_array = c.tuned_us;
    info->chunk_bytes = c.chunk_bytes;
    return BDCT_OK;
}
