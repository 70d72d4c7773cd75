// batch.cu - batched solves (stag_batch_*): many independent systems
// A_k x_k = b_k advanced together.
//
// Systems with the same gauge field (same pointers, extents and mass) form a
// group and run as right-hand sides of multi-RHS Dirac kernels (every link is
// loaded once for a block of right-hand sides); groups of different lattice
// sizes share each launch through the work-item table of multi.cu.  The inner
// iteration is the mixed-precision CG of blas_lo.cu - FP32 vectors and links,
// FP64 scalars - and each right-hand side gets its own reliable updates: its
// iterated residual is replaced by the true residual b - A x computed in
// float-float arithmetic, and its final residual is confirmed in native FP64.
// The replacements are decided and applied on the device by a pass that
// follows every iteration (batch_dev.cu).  A block of check_interval
// iterations, each with its pass, is captured as one CUDA graph and replayed
// until the pass reports that no system is running; the host reads that one
// word between replays and does no per-system work.
//
// Autotuner: for each multi-RHS group the right-hand sides per thread
// (1, 2, 4, 8) and the threads per block (64, 128, 256) are timed on the
// group's own D_oe launch and the fastest is kept; single-RHS groups are tuned
// together over the block size.  Results are cached per (extents, Naik, RHS
// count) for the process, and in the file named by STAG_AUTOTUNE_CACHE if set.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/stag.h"
#include "handle.h"
#include "multi.cuh"

using namespace stag;

namespace stag {
void set_noalloc_error(const std::string& msg);  // thread-local message of stag_last_error(NULL)
static_assert(STAG_STATUS_OK == STAG_OK && STAG_STATUS_NOT_CONVERGED == STAG_ERR_NOT_CONVERGED &&
                  STAG_STATUS_BREAKDOWN == STAG_ERR_BREAKDOWN,
              "system statuses are the ABI's status codes");
}

namespace {

struct BFail {
    int code;
};

struct Tune {
    int rb = 1, bs = 256;
    double ms = 0.0;     // D_oe per launch
    double ms_eo = 0.0;  // reducing D_eo per launch (the candidate with the least D_oe + D_eo wins)
    int mode = 0;  // tile traversal (multi.cu): 0 contiguous runs, 1 resident sweep
};

struct Group {
    Geom g{};
    const double* fat_src = nullptr;
    const double* lng_src = nullptr;
    double mass = 0.0;
    int nrhs = 0, rpad = 1, rhs0 = 0, prhs0 = 0;
    double2 *fat64 = nullptr, *lng64 = nullptr;
    float4 *fatff = nullptr, *lngff = nullptr;
    float2 *fat32 = nullptr, *lng32 = nullptr;
    float2 *d = nullptr, *t = nullptr, *ad = nullptr, *r = nullptr, *y = nullptr;
    Tune tune;
    std::vector<int> systems;  // system index of each right-hand side
};

std::mutex g_tune_mu;
std::map<std::string, Tune> g_tune_cache;
bool g_tune_file_loaded = false;

}  // namespace

struct stag_batch {
    int n_sys = 0;
    int device = 0;
    stag_options opt{};
    cudaStream_t user_stream = nullptr, s = nullptr;
    cudaEvent_t ev_in = nullptr;
    std::vector<Group> groups;
    std::vector<int> sys_group, sys_slot;  // group and slot of each system (= right-hand side)
    std::vector<double2*> x64, b64;
    double2* r64 = nullptr;   // scratch, largest lattice
    double* io_a = nullptr;   // ABI staging, largest lattice
    double* io_b = nullptr;
    MultiGroup* d_groups = nullptr;
    int4* d_items = nullptr;
    std::vector<std::pair<Tune, std::pair<int, int>>> classes;  // (tuning, [first item, count))
    CgScalars* scal = nullptr;       // one per system
    CgScalars* aux = nullptr;        // scratch reductions
    CgScalars* scal_host = nullptr;  // pinned, n_sys + 1
    double* partials = nullptr;
    unsigned int* counters = nullptr;
    int max_blocks = 0;
    cudaGraphExec_t graph = nullptr;
    long long device_bytes = 0;
    std::string err = "no error";
    // device-side reliable updates (batch_dev.cu)
    std::vector<float4*> sys_scratch;      // per system: u_ff, t_ff, ax
    SysDev* d_sys = nullptr;
    SysState* d_state = nullptr;
    std::vector<SysState> state_host;
    SysDirac *d_oe_ff = nullptr, *d_eo_ff = nullptr, *d_oe_64 = nullptr, *d_eo_64 = nullptr;
    int* d_lists = nullptr;                // four lists: count, systems, tile prefix
    double* pass_partials = nullptr;       // one per tile of all systems
    int* running_host = nullptr;           // host-mapped count of running systems
    int* running_dev = nullptr;
    PassArgs pass{};
    int grid_dirac = 0, grid_vec = 0;
};

namespace {

void bfail(stag_batch* b, int code, const std::string& msg) {
    if (b) b->err = msg;
    set_noalloc_error(msg);
    throw BFail{code};
}

void bcheck(stag_batch* b, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    bfail(b, e == cudaErrorMemoryAllocation ? STAG_ERR_OOM : STAG_ERR_CUDA,
          std::string(what) + ": " + cudaGetErrorString(e));
}

template <class T>
T* balloc(stag_batch* b, size_t bytes, const char* what) {
    void* p = nullptr;
    bcheck(b, cudaMalloc(&p, bytes), what);
    b->device_bytes += (long long)bytes;
    bcheck(b, cudaMemsetAsync(p, 0, bytes, b->s), what);
    return static_cast<T*>(p);
}

bool on_dev(stag_batch* b, const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice && a.device != b->device)
        bfail(b, STAG_ERR_INVALID_ARG, "device pointer belongs to another device");
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void sync(stag_batch* b) { bcheck(b, cudaStreamSynchronize(b->s), "cudaStreamSynchronize"); }

size_t vec_bytes(const Geom& g) { return (size_t)3 * g.vs * sizeof(double2); }
size_t abi_bytes(const Geom& g) { return (size_t)3 * g.vh * sizeof(double2); }


void pack_group_field(stag_batch* b, Group& G, const double* src, double2* s64, float4* sff, float2* s32) {
    const size_t aos = (size_t)2 * G.g.vh * 4 * 9 * sizeof(double2);
    void* stage = nullptr;
    const double* p = src;
    if (!on_dev(b, src)) {
        bcheck(b, cudaMalloc(&stage, aos), "allocate link staging");
        cudaError_t e = cudaMemcpyAsync(stage, src, aos, cudaMemcpyHostToDevice, b->s);
        if (e != cudaSuccess) {
            cudaFree(stage);
            bcheck(b, e, "copy links");
        }
        p = static_cast<const double*>(stage);
    }
    launch_pack_links(G.g, p, s64, sff, s32, nullptr, nullptr, b->s);
    cudaError_t e = cudaGetLastError();
    if (stage) {
        const cudaError_t e2 = cudaStreamSynchronize(b->s);
        cudaFree(stage);
        if (e == cudaSuccess) e = e2;
    }
    bcheck(b, e, "pack links");
}

MultiLaunch make_launch(stag_batch* b, int parity, int phase, int first_item) {
    MultiLaunch L;
    L.groups = b->d_groups;
    L.items = b->d_items + first_item;
    L.scal = b->scal;
    L.partials = b->partials;
    L.counters = b->counters;
    L.out_parity = parity;
    L.phase = phase;
    return L;
}

// Blocks per group and launch (and partial-sum capacity).  Each block ends with
// a per-right-hand-side reduction, so fewer, longer blocks (contiguous runs of
// tiles) pay less for them: 16 RHS at 32^3 x 64 take 3.97 s with one tile per
// block (16384 blocks), 3.48 s with 4096 blocks and 3.60 s with 2048.
constexpr int kMaxGroupBlocks = 4096;

// Blocks of a group for a shape: one per tile of sites, at most kMaxGroupBlocks
// (blocks then take contiguous runs of tiles); for the resident sweep, at most
// the number of blocks of that shape the GPU holds at once.
int group_blocks(const Group& G, int rb, int bs, int mode) {
    const int spb = bs / (G.rpad / rb);
    const int ntiles = (G.g.vh + spb - 1) / spb;
    int cap = kMaxGroupBlocks;
    if (mode) {
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cap = std::min(cap, multi_resident_blocks_per_sm(rb, bs) * sms);
    }
    return std::min(ntiles, cap);
}

void add_items(std::vector<int4>& v, int gi, int nblk, int mode) {
    for (int k = 0; k < nblk; ++k) v.push_back(make_int4(gi, k, nblk, mode));
}

// Work items of every group with its tuned shape, grouped into launch classes.
void build_items(stag_batch* b) {
    std::map<std::tuple<int, int, int>, std::vector<int4>> by_class;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const Group& G = b->groups[gi];
        add_items(by_class[{G.tune.rb, G.tune.bs, G.tune.mode}], (int)gi,
                  group_blocks(G, G.tune.rb, G.tune.bs, G.tune.mode), G.tune.mode);
    }
    std::vector<int4> all;
    b->classes.clear();
    for (auto& kv : by_class) {
        Tune t;
        t.rb = std::get<0>(kv.first);
        t.bs = std::get<1>(kv.first);
        t.mode = std::get<2>(kv.first);
        b->classes.push_back({t, {(int)all.size(), (int)kv.second.size()}});
        all.insert(all.end(), kv.second.begin(), kv.second.end());
    }
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    bcheck(b, cudaMalloc(&b->d_items, std::max<size_t>(1, all.size()) * sizeof(int4)), "allocate work items");
    bcheck(b, cudaMemcpyAsync(b->d_items, all.data(), all.size() * sizeof(int4), cudaMemcpyHostToDevice, b->s),
           "copy work items");
    sync(b);
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
}

void enqueue_all(stag_batch* b, MultiKernel k, int parity, int phase) {
    for (auto& c : b->classes)
        launch_multi(k, make_launch(b, parity, phase, c.second.first), c.second.second, c.first.rb, c.first.bs,
                     c.first.mode, b->s);
}

void enqueue_iteration(stag_batch* b) {
    enqueue_all(b, MK_DSLASH_PLAIN, 1, 0);
    enqueue_all(b, MK_DSLASH_CG, 0, 1);
    enqueue_all(b, MK_UPDATE_XR, 0, 0);
    enqueue_all(b, MK_UPDATE_D, 0, 0);
}

// ------------------------------------------------------------ autotuner
std::string tune_key(const Group& G) {
    std::ostringstream os;
    os << G.g.lx << "x" << G.g.ly << "x" << G.g.lz << "x" << G.g.lt << (G.lng_src ? ":naik" : ":onehop") << ":"
       << G.nrhs;
    return os.str();
}

void load_tune_file() {
    if (g_tune_file_loaded) return;
    g_tune_file_loaded = true;
    const char* path = std::getenv("STAG_AUTOTUNE_CACHE");
    if (!path) return;
    std::ifstream f(path);
    std::string key;
    // lines: key rb bs ms [traversal]
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream ls(line);
        Tune t;
        if (ls >> key >> t.rb >> t.bs >> t.ms) {
            if (!(ls >> t.mode)) t.mode = 0;
            g_tune_cache[key] = t;
        }
    }
}

// Every candidate's time, appended to the file STAG_AUTOTUNE_LOG names (if set).
void log_candidate(const std::string& key, int rb, int bs, int mode, double ms_oe, double ms_eo) {
    if (const char* path = std::getenv("STAG_AUTOTUNE_LOG")) {
        std::ofstream f(path, std::ios::app);
        f << key << " rb=" << rb << " bs=" << bs << " traversal=" << mode << " ms_oe=" << ms_oe << " ms_eo=" << ms_eo
          << "\n";
    }
}

void store_tune(const std::string& key, const Tune& t) {
    g_tune_cache[key] = t;
    if (const char* path = std::getenv("STAG_AUTOTUNE_CACHE")) {
        std::ofstream f(path, std::ios::app);
        f << key << " " << t.rb << " " << t.bs << " " << t.ms << " " << t.mode << "\n";
    }
}

// Best of three timed launches (after a warm-up) of the group's D_oe and of
// its reducing D_eo (the two Dirac launches of every iteration), in ms.  The
// CG state is cleared before each launch so that it does its full work (with
// zero vectors the D_eo epilogue marks the systems done, and a launch for a
// group whose systems are all done returns at once).
std::pair<double, double> time_group_launch(stag_batch* b, const std::vector<int>& gis, int rb, int bs, int mode) {
    std::vector<int4> items;
    for (int gi : gis) add_items(items, gi, group_blocks(b->groups[gi], rb, bs, mode), mode);
    int4* d_items = nullptr;
    bcheck(b, cudaMalloc(&d_items, items.size() * sizeof(int4)), "allocate tuning items");
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // D_oe start, end; D_eo start, end
    double best_oe = 1e30, best_eo = 1e30;
    cudaError_t err = cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, b->s);
    for (int k = 0; k < 4 && err == cudaSuccess; ++k) err = cudaEventCreate(&ev[k]);
    MultiLaunch L;
    L.groups = b->d_groups;
    L.items = d_items;
    L.scal = b->scal;
    L.partials = b->partials;
    L.counters = b->counters;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
        // a cleared state: no system is done, so every launch does its full work
        err = cudaMemsetAsync(b->scal, 0, sizeof(CgScalars) * b->n_sys, b->s);
        if (err != cudaSuccess) break;
        L.out_parity = 1;
        L.phase = 0;
        cudaEventRecord(ev[0], b->s);
        launch_multi(MK_DSLASH_PLAIN, L, (int)items.size(), rb, bs, mode, b->s);
        cudaEventRecord(ev[1], b->s);
        err = cudaMemsetAsync(b->scal, 0, sizeof(CgScalars) * b->n_sys, b->s);
        if (err != cudaSuccess) break;
        L.out_parity = 0;
        L.phase = 1;
        cudaEventRecord(ev[2], b->s);
        launch_multi(MK_DSLASH_CG, L, (int)items.size(), rb, bs, mode, b->s);
        cudaEventRecord(ev[3], b->s);
        err = cudaEventSynchronize(ev[3]);
        float ms_oe = 0.f, ms_eo = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms_oe, ev[0], ev[1]);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms_eo, ev[2], ev[3]);
        if (rep > 0) {  // the first launches are a warm-up
            best_oe = std::min(best_oe, (double)ms_oe);
            best_eo = std::min(best_eo, (double)ms_eo);
        }
    }
    if (err == cudaSuccess) err = cudaMemsetAsync(b->scal, 0, sizeof(CgScalars) * b->n_sys, b->s);
    if (err == cudaSuccess) err = cudaGetLastError();
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    cudaFree(d_items);
    bcheck(b, err, "autotune");
    return {best_oe, best_eo};
}

void autotune(stag_batch* b) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_tune_file();
    const bool enabled = b->opt.autotune != 0;
    std::vector<int> singles;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        Group& G = b->groups[gi];
        if (G.nrhs == 1) {
            singles.push_back((int)gi);
            continue;
        }
        const std::string key = tune_key(G);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            G.tune = it->second;
            continue;
        }
        Tune best;
        best.rb = std::max(std::min(4, G.rpad), G.rpad / 32);
        best.bs = 128;
        double best_pair = 1e30;
        if (enabled) {
            for (int mode : {0, 1}) {
                for (int rb : {1, 2, 4, 8}) {
                    if (rb > G.rpad || G.rpad / rb > 32) continue;
                    for (int bs : {64, 128, 256}) {
                        const auto t = time_group_launch(b, {(int)gi}, rb, bs, mode);
                        log_candidate(key, rb, bs, mode, t.first, t.second);
                        if (t.first + t.second < best_pair) {
                            best_pair = t.first + t.second;
                            best.ms = t.first;
                            best.ms_eo = t.second;
                            best.rb = rb;
                            best.bs = bs;
                            best.mode = mode;
                        }
                    }
                }
            }
            store_tune(key, best);
        }
        G.tune = best;
    }
    if (!singles.empty()) {
        Tune best;
        best.rb = 1;
        best.bs = 128;
        double best_pair = 1e30;
        if (enabled) {
            for (int mode : {0, 1}) {
                for (int bs : {64, 128, 256}) {
                    const auto t = time_group_launch(b, singles, 1, bs, mode);
                    log_candidate("single-rhs", 1, bs, mode, t.first, t.second);
                    if (t.first + t.second < best_pair) {
                        best_pair = t.first + t.second;
                        best.ms = t.first;
                        best.ms_eo = t.second;
                        best.bs = bs;
                        best.mode = mode;
                    }
                }
            }
        }
        for (int gi : singles) b->groups[gi].tune = best;
    }
}

// ------------------------------------------------------- reliable update
double read_aux(stag_batch* b) {
    bcheck(b, cudaMemcpyAsync(b->scal_host + b->n_sys, b->aux, sizeof(CgScalars), cudaMemcpyDeviceToHost, b->s),
           "read reduction");
    sync(b);
    return b->scal_host[b->n_sys].red_out;
}

void destroy_batch(stag_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->s) cudaStreamSynchronize(b->s);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (Group& G : b->groups) {
        for (void* p : {(void*)G.fat64, (void*)G.lng64, (void*)G.fatff, (void*)G.lngff, (void*)G.fat32,
                        (void*)G.lng32, (void*)G.d, (void*)G.t, (void*)G.ad, (void*)G.r, (void*)G.y})
            if (p) cudaFree(p);
    }
    for (double2* p : b->x64)
        if (p) cudaFree(p);
    for (double2* p : b->b64)
        if (p) cudaFree(p);
    for (void* p : {(void*)b->r64, (void*)b->io_a, (void*)b->io_b, (void*)b->d_groups, (void*)b->d_items,
                    (void*)b->scal, (void*)b->aux, (void*)b->partials, (void*)b->counters, (void*)b->d_sys,
                    (void*)b->d_state, (void*)b->d_oe_ff, (void*)b->d_eo_ff, (void*)b->d_oe_64, (void*)b->d_eo_64,
                    (void*)b->d_lists, (void*)b->pass_partials})
        if (p) cudaFree(p);
    for (float4* p : b->sys_scratch)
        if (p) cudaFree(p);
    if (b->running_host) cudaFreeHost(b->running_host);
    if (b->scal_host) cudaFreeHost(b->scal_host);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->s) cudaStreamDestroy(b->s);
    delete b;
}

// Per-system operands and scratch of the device-side reliable updates, the
// device lists, and the host-mapped running count (batch_dev.cu).
void setup_pass(stag_batch* b) {
    const int n = b->n_sys;
    std::vector<SysDev> sd(n);
    std::vector<SysDirac> oe_ff(n), eo_ff(n), oe_64(n), eo_64(n);
    long long tiles = 0;
    b->sys_scratch.assign(3 * (size_t)n, nullptr);
    for (int k = 0; k < n; ++k) {
        Group& G = b->groups[b->sys_group[k]];
        const Geom& g = G.g;
        float4* u = balloc<float4>(b, vec_bytes(g), "allocate reliable-update scratch");
        b->sys_scratch[3 * k] = u;
        float4* t = balloc<float4>(b, vec_bytes(g), "allocate reliable-update scratch");
        b->sys_scratch[3 * k + 1] = t;
        float4* ax = balloc<float4>(b, vec_bytes(g), "allocate reliable-update scratch");
        b->sys_scratch[3 * k + 2] = ax;
        const double m2 = G.mass * G.mass;
        sd[k] = SysDev{g, m2, b->x64[k], b->b64[k], u, t, ax, G.r, G.d, G.y, G.rpad, b->sys_slot[k]};
        const float2 m2ff = host_ff_from_double(m2);
        oe_ff[k] = SysDirac{g, 1, G.fatff, G.lngff, u, t, nullptr, 0.0, make_float2(0.f, 0.f)};
        eo_ff[k] = SysDirac{g, 0, G.fatff, G.lngff, t, ax, u, m2, m2ff};
        oe_64[k] = SysDirac{g, 1, G.fat64, G.lng64, b->x64[k], t, nullptr, 0.0, make_float2(0.f, 0.f)};
        eo_64[k] = SysDirac{g, 0, G.fat64, G.lng64, t, ax, b->x64[k], m2, m2ff};
        tiles += (g.vh + kBlock - 1) / kBlock;
    }
    b->d_sys = balloc<SysDev>(b, sizeof(SysDev) * n, "allocate systems");
    b->d_state = balloc<SysState>(b, sizeof(SysState) * n, "allocate systems");
    b->d_oe_ff = balloc<SysDirac>(b, sizeof(SysDirac) * n, "allocate systems");
    b->d_eo_ff = balloc<SysDirac>(b, sizeof(SysDirac) * n, "allocate systems");
    b->d_oe_64 = balloc<SysDirac>(b, sizeof(SysDirac) * n, "allocate systems");
    b->d_eo_64 = balloc<SysDirac>(b, sizeof(SysDirac) * n, "allocate systems");
    bcheck(b, cudaMemcpyAsync(b->d_sys, sd.data(), sizeof(SysDev) * n, cudaMemcpyHostToDevice, b->s), "copy systems");
    bcheck(b, cudaMemcpyAsync(b->d_oe_ff, oe_ff.data(), sizeof(SysDirac) * n, cudaMemcpyHostToDevice, b->s), "copy");
    bcheck(b, cudaMemcpyAsync(b->d_eo_ff, eo_ff.data(), sizeof(SysDirac) * n, cudaMemcpyHostToDevice, b->s), "copy");
    bcheck(b, cudaMemcpyAsync(b->d_oe_64, oe_64.data(), sizeof(SysDirac) * n, cudaMemcpyHostToDevice, b->s), "copy");
    bcheck(b, cudaMemcpyAsync(b->d_eo_64, eo_64.data(), sizeof(SysDirac) * n, cudaMemcpyHostToDevice, b->s), "copy");
    // four lists of 1 + n + (n + 1) ints
    const size_t per_list = 2 * (size_t)n + 2;
    b->d_lists = balloc<int>(b, sizeof(int) * 4 * per_list, "allocate lists");
    PassList* lists[4] = {&b->pass.fold, &b->pass.ff, &b->pass.confirm, &b->pass.replace};
    for (int q = 0; q < 4; ++q) {
        int* base = b->d_lists + q * per_list;
        *lists[q] = PassList{base, base + 1, base + 1 + n};
    }
    b->pass_partials = balloc<double>(b, sizeof(double) * (size_t)std::max<long long>(1, tiles), "allocate partials");
    bcheck(b, cudaHostAlloc(reinterpret_cast<void**>(&b->running_host), sizeof(int), cudaHostAllocMapped),
           "allocate mapped count");
    *b->running_host = 0;
    bcheck(b, cudaHostGetDevicePointer(reinterpret_cast<void**>(&b->running_dev), b->running_host, 0),
           "map count");
    b->pass.n_sys = n;
    b->pass.sys = b->d_sys;
    b->pass.state = b->d_state;
    b->pass.scal = b->scal;
    b->pass.partials = b->pass_partials;
    b->pass.running = b->running_dev;
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    b->grid_dirac = 3 * sms;
    b->grid_vec = 8 * sms;
    b->state_host.assign(n, SysState{});
}

void enqueue_pass(stag_batch* b) {
    enqueue_reliable_pass(b->pass, b->d_oe_ff, b->d_eo_ff, b->d_oe_64, b->d_eo_64, b->grid_dirac, b->grid_vec,
                          b->s);
}

void begin(stag_batch* b) {
    bcheck(b, cudaSetDevice(b->device), "cudaSetDevice");
    bcheck(b, cudaEventRecord(b->ev_in, b->user_stream), "cudaEventRecord");
    bcheck(b, cudaStreamWaitEvent(b->s, b->ev_in, 0), "cudaStreamWaitEvent");
}

}  // namespace

extern "C" {

int stag_batch_create(stag_batch** out, int32_t n_sys, const double* const* fat, const double* const* naik,
                      const int32_t* dims, const double* masses, const stag_options* opt) {
    if (out) *out = nullptr;
    stag_batch* b = nullptr;
    try {
        if (!out || !fat || !dims || !masses || n_sys < 1)
            bfail(nullptr, STAG_ERR_INVALID_ARG, "stag_batch_create: bad arguments");
        b = new stag_batch();
        b->n_sys = n_sys;
        stag_default_options(&b->opt);
        // Replacements happen on the device after every iteration, so the
        // interval only sets how often the host looks at the running count (and
        // how many empty iterations can follow the last system's convergence).
        b->opt.check_interval = 8;
        if (opt) b->opt = *opt;
        if (b->opt.check_interval < 1 || b->opt.check_interval > 4096)
            bfail(b, STAG_ERR_INVALID_ARG, "check_interval must be in [1, 4096]");
        if (b->opt.reliable_interval < 1 || !(b->opt.reliable_delta > 0.0 && b->opt.reliable_delta < 1.0))
            bfail(b, STAG_ERR_INVALID_ARG, "reliable_interval must be >= 1 and reliable_delta in (0, 1)");
        if (b->opt.link_recon != 0 || b->opt.long_recon != 0)
            bfail(b, STAG_ERR_INVALID_ARG, "batches keep all nine link entries (link_recon = long_recon = 0)");
        bcheck(b, cudaGetDevice(&b->device), "cudaGetDevice");
        bcheck(b, cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking), "cudaStreamCreate");
        bcheck(b, cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming), "cudaEventCreate");
        begin(b);
        // group the systems
        b->sys_group.assign(n_sys, -1);
        b->sys_slot.assign(n_sys, 0);
        for (int k = 0; k < n_sys; ++k) {
            const int32_t* dk = dims + 4 * k;
            long long V = 1;
            for (int m = 0; m < 4; ++m) {
                if (dk[m] < 2 || dk[m] % 2) bfail(b, STAG_ERR_INVALID_ARG, "every lattice extent must be even and >= 2");
                V *= dk[m];
            }
            if (V / 2 >= (1LL << 30)) bfail(b, STAG_ERR_INVALID_ARG, "lattice too large");
            if (!fat[k]) bfail(b, STAG_ERR_INVALID_ARG, "NULL links");
            if (!std::isfinite(masses[k])) bfail(b, STAG_ERR_INVALID_ARG, "mass must be finite");
            const double* nk = naik ? naik[k] : nullptr;
            int gi = -1;
            for (size_t q = 0; q < b->groups.size(); ++q) {
                const Group& G = b->groups[q];
                if (G.fat_src == fat[k] && G.lng_src == nk && G.mass == masses[k] && G.g.lx == dk[0] &&
                    G.g.ly == dk[1] && G.g.lz == dk[2] && G.g.lt == dk[3])
                    gi = (int)q;
            }
            if (gi < 0) {
                Group G;
                G.g.lx = dk[0];
                G.g.ly = dk[1];
                G.g.lz = dk[2];
                G.g.lt = dk[3];
                G.g.lxh = dk[0] / 2;
                G.g.vh = (int)(V / 2);
                G.g.vs = (int)((V / 2 + 63) / 64 * 64);
                for (int m = 0; m < 4; ++m) G.g.hop3[m] = 3 % dk[m];
                G.fat_src = fat[k];
                G.lng_src = nk;
                G.mass = masses[k];
                b->groups.push_back(G);
                gi = (int)b->groups.size() - 1;
            }
            b->sys_group[k] = gi;
            b->sys_slot[k] = b->groups[gi].nrhs++;
            b->groups[gi].systems.push_back(k);
        }
        // allocate and pack
        size_t max_vs = 0, max_vh = 0;
        int rhs0 = 0, prhs0 = 0;
        std::vector<MultiGroup> mg;
        for (Group& G : b->groups) {
            if (G.nrhs > 256) bfail(b, STAG_ERR_INVALID_ARG, "at most 256 right-hand sides share one field");
            G.rpad = 1;
            while (G.rpad < G.nrhs) G.rpad *= 2;  // power of two: rpad / rb lanes divide a warp
            if (G.nrhs > 1) G.rpad = std::max(G.rpad, 8);
            G.rhs0 = rhs0;
            rhs0 += G.nrhs;
            G.prhs0 = prhs0;
            prhs0 += G.rpad;
            max_vs = std::max(max_vs, (size_t)G.g.vs);
            max_vh = std::max(max_vh, (size_t)G.g.vh);
            b->max_blocks = kMaxGroupBlocks;
            const size_t nl = (size_t)2 * 4 * 9 * G.g.vs;
            G.fat64 = balloc<double2>(b, nl * sizeof(double2), "allocate links");
            G.fatff = balloc<float4>(b, nl * sizeof(float4), "allocate links");
            G.fat32 = balloc<float2>(b, nl * sizeof(float2), "allocate links");
            pack_group_field(b, G, G.fat_src, G.fat64, G.fatff, G.fat32);
            if (G.lng_src) {
                G.lng64 = balloc<double2>(b, nl * sizeof(double2), "allocate links");
                G.lngff = balloc<float4>(b, nl * sizeof(float4), "allocate links");
                G.lng32 = balloc<float2>(b, nl * sizeof(float2), "allocate links");
                pack_group_field(b, G, G.lng_src, G.lng64, G.lngff, G.lng32);
            }
            const size_t vb = (size_t)3 * G.g.vs * G.rpad * sizeof(float2);
            G.d = balloc<float2>(b, vb, "allocate vectors");
            G.t = balloc<float2>(b, vb, "allocate vectors");
            G.ad = balloc<float2>(b, vb, "allocate vectors");
            G.r = balloc<float2>(b, vb, "allocate vectors");
            G.y = balloc<float2>(b, vb, "allocate vectors");
            MultiGroup m{G.g, G.fat32, G.lng32, G.d, G.t, G.ad, G.r, G.y, G.mass * G.mass, G.nrhs, G.rpad, G.rhs0,
                         G.prhs0, 0};
            mg.push_back(m);
        }
        for (auto& m : mg) m.max_blocks = b->max_blocks;
        b->x64.assign(n_sys, nullptr);
        b->b64.assign(n_sys, nullptr);
        for (int k = 0; k < n_sys; ++k) {
            const Geom& g = b->groups[b->sys_group[k]].g;
            b->x64[k] = balloc<double2>(b, vec_bytes(g), "allocate x");
            b->b64[k] = balloc<double2>(b, vec_bytes(g), "allocate b");
        }
        const size_t vbmax = (size_t)3 * max_vs * sizeof(double2);
        b->r64 = balloc<double2>(b, vbmax, "allocate scratch");
        b->io_a = balloc<double>(b, (size_t)3 * max_vh * sizeof(double2), "allocate staging");
        b->io_b = balloc<double>(b, (size_t)3 * max_vh * sizeof(double2), "allocate staging");
        b->scal = balloc<CgScalars>(b, sizeof(CgScalars) * n_sys, "allocate CG state");
        b->aux = balloc<CgScalars>(b, sizeof(CgScalars), "allocate CG state");
        b->partials = balloc<double>(b, sizeof(double) * (size_t)prhs0 * b->max_blocks, "allocate partials");
        b->counters = balloc<unsigned int>(b, sizeof(unsigned int) * prhs0, "allocate counters");
        b->d_groups = balloc<MultiGroup>(b, sizeof(MultiGroup) * mg.size(), "allocate groups");
        bcheck(b, cudaMemcpyAsync(b->d_groups, mg.data(), sizeof(MultiGroup) * mg.size(), cudaMemcpyHostToDevice, b->s),
               "copy groups");
        bcheck(b, cudaMallocHost(reinterpret_cast<void**>(&b->scal_host), sizeof(CgScalars) * (n_sys + 1)),
               "allocate pinned state");
        std::memset(b->scal_host, 0, sizeof(CgScalars) * (n_sys + 1));
        setup_pass(b);
        sync(b);
        autotune(b);
        build_items(b);
        *out = b;
        return STAG_OK;
    } catch (const BFail& f) {
        destroy_batch(b);
        return f.code;
    } catch (...) {
        set_noalloc_error("unexpected exception");
        destroy_batch(b);
        return STAG_ERR_CUDA;
    }
}

int stag_batch_set_stream(stag_batch* b, void* cuda_stream) {
    if (!b) return STAG_ERR_INVALID_ARG;
    b->user_stream = static_cast<cudaStream_t>(cuda_stream);
    return STAG_OK;
}

int stag_batch_tuning(const stag_batch* b, int32_t system, int32_t* rhs_per_thread, int32_t* threads_per_block,
                      double* ms, int32_t* traversal) {
    if (!b || system < 0 || system >= b->n_sys) return STAG_ERR_INVALID_ARG;
    const Group& G = b->groups[b->sys_group[system]];
    if (rhs_per_thread) *rhs_per_thread = G.tune.rb;
    if (threads_per_block) *threads_per_block = G.tune.bs;
    if (ms) *ms = G.tune.ms;
    if (traversal) *traversal = G.tune.mode;
    return STAG_OK;
}

int stag_batch_set_tuning(stag_batch* b, int32_t system, int32_t rhs_per_thread, int32_t threads_per_block,
                          int32_t traversal) {
    if (!b) return STAG_ERR_INVALID_ARG;
    try {
        if (system < 0 || system >= b->n_sys) bfail(b, STAG_ERR_INVALID_ARG, "system index out of range");
        Group& G = b->groups[b->sys_group[system]];
        const int rb = rhs_per_thread, bs = threads_per_block;
        const bool rb_ok = (rb == 1 || rb == 2 || rb == 4 || rb == 8) && rb <= G.rpad && G.rpad / rb <= 32 &&
                           (G.nrhs > 1 || rb == 1);
        if (!rb_ok || (bs != 64 && bs != 128 && bs != 256) || (traversal != 0 && traversal != 1))
            bfail(b, STAG_ERR_INVALID_ARG, "stag_batch_set_tuning: unsupported shape");
        bcheck(b, cudaSetDevice(b->device), "cudaSetDevice");
        G.tune.rb = rb;
        G.tune.bs = bs;
        G.tune.mode = traversal;
        G.tune.ms = 0.0;
        build_items(b);
        return STAG_OK;
    } catch (const BFail& f) {
        return f.code;
    } catch (...) {
        b->err = "unexpected exception";
        return STAG_ERR_CUDA;
    }
}

int stag_batch_apply_A(stag_batch* b, const double* const* in, double* const* out) {
    if (!b) return STAG_ERR_INVALID_ARG;
    try {
        if (!in || !out) bfail(b, STAG_ERR_INVALID_ARG, "NULL argument");
        begin(b);
        // load every system's input into its slot of d, with all systems live
        bcheck(b, cudaMemsetAsync(b->scal, 0, sizeof(CgScalars) * b->n_sys, b->s), "clear CG state");
        for (int k = 0; k < b->n_sys; ++k) {
            Group& G = b->groups[b->sys_group[k]];
            const double* src = in[k];
            if (!src || !out[k]) bfail(b, STAG_ERR_INVALID_ARG, "NULL vector");
            if (!on_dev(b, src)) {
                bcheck(b, cudaMemcpyAsync(b->io_a, src, abi_bytes(G.g), cudaMemcpyHostToDevice, b->s), "copy input");
                src = b->io_a;
            }
            launch_pack_vec(G.g, src, b->r64, b->s);
            launch_slot_put(G.g, b->r64, G.d, G.rpad, b->sys_slot[k], b->s);
        }
        enqueue_all(b, MK_DSLASH_PLAIN, 1, 0);
        enqueue_all(b, MK_DSLASH_AXPY, 0, 1);
        for (int k = 0; k < b->n_sys; ++k) {
            Group& G = b->groups[b->sys_group[k]];
            launch_slot_get(G.g, G.ad, b->r64, G.rpad, b->sys_slot[k], b->s);
            const bool dev = on_dev(b, out[k]);
            launch_unpack_vec(G.g, b->r64, dev ? out[k] : b->io_b, b->s);
            if (!dev)
                bcheck(b, cudaMemcpyAsync(out[k], b->io_b, abi_bytes(G.g), cudaMemcpyDeviceToHost, b->s), "copy output");
            sync(b);
        }
        bcheck(b, cudaGetLastError(), "batch apply_A");
        sync(b);
        return STAG_OK;
    } catch (const BFail& f) {
        return f.code;
    } catch (...) {
        b->err = "unexpected exception";
        return STAG_ERR_CUDA;
    }
}

int stag_batch_solve(stag_batch* b, const double* const* bvec, double* const* xvec, double tol, int32_t max_iter,
                     stag_solve_info* infos) {
    if (!b) return STAG_ERR_INVALID_ARG;
    NvtxRange range("stag_batch_solve");
    const int n = b->n_sys;
    std::vector<stag_solve_info> inf(n);
    int status = STAG_OK;
    const auto t0 = std::chrono::steady_clock::now();
    try {
        if (!bvec || !xvec) bfail(b, STAG_ERR_INVALID_ARG, "NULL argument");
        if (!(tol > 0.0) || !std::isfinite(tol)) bfail(b, STAG_ERR_INVALID_ARG, "tol must be positive and finite");
        begin(b);
        const long long max_it = max_iter > 0 ? max_iter : (1LL << 40);
        // every system idles (done = 1) until the first pass has set it up
        for (int k = 0; k < n; ++k) {
            std::memset(&b->scal_host[k], 0, sizeof(CgScalars));
            b->scal_host[k].done = 1;
        }
        for (int k = 0; k < n; ++k) {
            Group& G = b->groups[b->sys_group[k]];
            if (!bvec[k] || !xvec[k]) bfail(b, STAG_ERR_INVALID_ARG, "NULL vector");
            const double* bs = bvec[k];
            if (!on_dev(b, bs)) {
                bcheck(b, cudaMemcpyAsync(b->io_a, bs, abi_bytes(G.g), cudaMemcpyHostToDevice, b->s), "copy b");
                bs = b->io_a;
            }
            launch_pack_vec(G.g, bs, b->b64[k], b->s);
            const double* xs = xvec[k];
            if (!on_dev(b, xs)) {
                bcheck(b, cudaMemcpyAsync(b->io_b, xs, abi_bytes(G.g), cudaMemcpyHostToDevice, b->s), "copy x");
                xs = b->io_b;
            }
            launch_pack_vec(G.g, xs, b->x64[k], b->s);
            launch_norm2_diff(G.g, b->b64[k], nullptr, b->aux, b->partials, b->s);
            const double bnorm2 = read_aux(b);
            if (!std::isfinite(bnorm2)) bfail(b, STAG_ERR_INVALID_ARG, "source has non-finite entries");
            SysState& st = b->state_host[k];
            st = SysState{};
            st.bnorm2 = bnorm2;
            st.tol = tol;
            st.tol2 = tol * tol * bnorm2;
            st.rel_delta = b->opt.reliable_delta;
            st.rel_interval = b->opt.reliable_interval;
            st.max_iter = max_it;
            st.first = 1;
            st.phase = SYS_START;
            if (bnorm2 == 0.0) {  // x = 0 solves it exactly
                bcheck(b, cudaMemsetAsync(b->x64[k], 0, vec_bytes(G.g), b->s), "zero x");
                st.phase = SYS_FINISHED;
                st.status = STAG_OK;
            }
        }
        bcheck(b, cudaMemcpyAsync(b->scal, b->scal_host, sizeof(CgScalars) * n, cudaMemcpyHostToDevice, b->s),
               "set CG state");
        bcheck(b, cudaMemcpyAsync(b->d_state, b->state_host.data(), sizeof(SysState) * n, cudaMemcpyHostToDevice,
                                  b->s),
               "set system state");
        *b->running_host = n;
        enqueue_pass(b);  // the first true residuals and replacements
        bcheck(b, cudaGetLastError(), "batch start");
        if (!b->graph) {
            // check_interval iterations of every group, each followed by the
            // reliable-update pass: a system due for a replacement waits at most
            // one iteration, and the host reads one word per graph launch
            cudaGraph_t graph = nullptr;
            bcheck(b, cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal), "begin capture");
            for (int it = 0; it < b->opt.check_interval; ++it) {
                enqueue_iteration(b);
                enqueue_pass(b);
            }
            const cudaError_t e = cudaStreamEndCapture(b->s, &graph);
            bcheck(b, e, "end capture");
            const cudaError_t e2 = cudaGraphInstantiate(&b->graph, graph, 0);
            cudaGraphDestroy(graph);
            bcheck(b, e2, "graph instantiate");
        }
        sync(b);
        while (*static_cast<volatile int*>(b->running_host) > 0) {
            bcheck(b, cudaGraphLaunch(b->graph, b->s), "cudaGraphLaunch");
            sync(b);
        }
        bcheck(b, cudaMemcpyAsync(b->state_host.data(), b->d_state, sizeof(SysState) * n, cudaMemcpyDeviceToHost,
                                  b->s),
               "read system state");
        sync(b);
        for (int k = 0; k < n; ++k) {
            Group& G = b->groups[b->sys_group[k]];
            const SysState& st = b->state_host[k];
            inf[k].iters = (int32_t)st.iters;
            inf[k].reliable_updates = st.updates;
            inf[k].true_rel_residual = st.rel;
            inf[k].iter_rel_residual = st.rel;
            inf[k].status = st.status;
            const bool dev = on_dev(b, xvec[k]);
            launch_unpack_vec(G.g, b->x64[k], dev ? xvec[k] : b->io_b, b->s);
            if (!dev)
                bcheck(b, cudaMemcpyAsync(xvec[k], b->io_b, abi_bytes(G.g), cudaMemcpyDeviceToHost, b->s), "copy x");
            sync(b);
            if (inf[k].status != STAG_OK && status == STAG_OK) status = inf[k].status;
        }
        bcheck(b, cudaGetLastError(), "batch solve");
    } catch (const BFail& f) {
        status = f.code;
    } catch (...) {
        b->err = "unexpected exception";
        status = STAG_ERR_CUDA;
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (infos) {
        for (int k = 0; k < n; ++k) {
            inf[k].time_ms = ms;
            if (inf[k].status == STAG_OK && status != STAG_OK && status != STAG_ERR_NOT_CONVERGED &&
                status != STAG_ERR_BREAKDOWN)
                inf[k].status = status;
            infos[k] = inf[k];
        }
    }
    return status;
}

const char* stag_batch_last_error(const stag_batch* b) { return b ? b->err.c_str() : stag_last_error(nullptr); }

int64_t stag_batch_device_bytes(const stag_batch* b) { return b ? b->device_bytes : 0; }

int stag_batch_destroy(stag_batch* b) {
    destroy_batch(b);
    return STAG_OK;
}

}  // extern "C"
