// batch.cu -- many independent pressure systems in one persistent cooperative
// launch (each system owns a contiguous range of blocks and converges on its
// own), replayed from a CUDA graph; plus the autotuner that picks the block
// size and the split of the grid between systems.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "solve.cuh"

namespace spuma {

SolveArgs make_args(spuma_ldu_t h);
void fill_controls(SolveArgs& a, const spuma_solver_controls* ctl);
bool ctl_ok(const spuma_solver_controls* c);
int solve_blocks_per_sm(int threads, bool batch, int kind, size_t dyn = 0);
int batch_kind(int precision);
spuma_status launch_batch_kernel(const BatchTable& t, int grid, int threads, int kind, cudaStream_t s);

// Split `grid` blocks between systems in proportion to their weights, at
// least one block each (largest-remainder rounding; deterministic).
bool batch_split(int n_sys, const double* w, int grid, int* split)
{
    if (n_sys <= 0 || grid < n_sys) return false;
    double tot = 0.0;
    for (int k = 0; k < n_sys; k++) tot += std::max(w[k], 0.0);
    std::vector<int> nb(n_sys, 1);
    int rest = grid - n_sys;
    std::vector<std::pair<double, int>> rem;
    int given = 0;
    for (int k = 0; k < n_sys; k++) {
        double share = tot > 0.0 ? rest * std::max(w[k], 0.0) / tot : (double)rest / n_sys;
        int fl = (int)std::floor(share);
        nb[k] += fl;
        given += fl;
        rem.push_back({share - fl, k});
    }
    std::stable_sort(rem.begin(), rem.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
        return a.first > b.first;
    });
    for (int j = 0; given < rest; j++, given++) nb[rem[j % n_sys].second]++;
    split[0] = 0;
    for (int k = 0; k < n_sys; k++) split[k + 1] = split[k] + nb[k];
    return split[n_sys] == grid;
}

// ------------------------------------------------------------ tune cache --
// A JSON object, one entry per line:  "signature": [threads, policy, grid_div, ms],
// (lines of the older three-number form read with grid_div 1).
static std::mutex g_tune_mu;
static std::map<std::string, std::vector<double>> g_tune_mem;

static bool parse_tune_line(const char* line, std::string& key, std::vector<double>& v)
{
    char k[768];
    double t = 0, p = 0, d = 0, m = 0;
    if (sscanf(line, " \"%767[^\"]\" : [ %lf , %lf , %lf , %lf ]", k, &t, &p, &d, &m) == 5) {
        key = k;
        v = {t, p, d, m};
        return true;
    }
    if (sscanf(line, " \"%767[^\"]\" : [ %lf , %lf , %lf ]", k, &t, &p, &m) == 4) {
        key = k;
        v = {t, p, 1.0, m};
        return true;
    }
    return false;
}

static void read_tune_file(const char* path, std::map<std::string, std::vector<double>>& into)
{
    FILE* f = fopen(path, "r");
    if (!f) return;
    char line[1024];
    std::string key;
    std::vector<double> v;
    while (fgets(line, sizeof line, f))
        if (parse_tune_line(line, key, v)) into[key] = v;
    fclose(f);
}

bool tune_cache_lookup(const char* path, const std::string& sig, int* threads, int* policy, int* grid_div, double* ms)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_mem.find(sig);
    if (it == g_tune_mem.end() && path && *path) {
        read_tune_file(path, g_tune_mem);
        it = g_tune_mem.find(sig);
    }
    if (it == g_tune_mem.end()) return false;
    *threads = (int)it->second[0];
    *policy = (int)it->second[1];
    *grid_div = std::max(1, (int)it->second[2]);
    *ms = it->second[3];
    return true;
}

bool tune_cache_store(const char* path, const std::string& sig, int threads, int policy, int grid_div, double ms)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const std::vector<double> val = {(double)threads, (double)policy, (double)grid_div, ms};
    g_tune_mem[sig] = val;
    if (!path || !*path) return true;
    std::map<std::string, std::vector<double>> all;
    read_tune_file(path, all);
    all[sig] = val;
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fprintf(f, "{\n");
    size_t k = 0;
    for (auto& e : all) {
        fprintf(f, "  \"%s\": [%d, %d, %d, %.6f]%s\n", e.first.c_str(), (int)e.second[0], (int)e.second[1],
                (int)e.second[2], e.second[3], ++k < all.size() ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    return std::rename(tmp.c_str(), path) == 0;
}

// Block weights per system: the cell count raised to 1 (policy 0), 4/3
// (policy 1: cells times an iteration count that grows like the mesh side)
// or 5/3 (policy 2: more blocks still to the large systems, whose solves are
// the longest).
constexpr int kPolicies = 3;
static void policy_weights(int policy, const std::vector<spuma_ldu_t>& hs, std::vector<double>& w)
{
    static const double expo[kPolicies] = {1.0, 4.0 / 3.0, 5.0 / 3.0};
    w.resize(hs.size());
    for (size_t k = 0; k < hs.size(); k++) {
        double n = std::max(1, hs[k]->n);
        w[k] = std::pow(n, expo[std::min(std::max(policy, 0), kPolicies - 1)]);
    }
}

}  // namespace spuma

using namespace spuma;

struct spuma_batch_trial {
    int threads, policy, grid_div, grid;
    double ms;
};

struct spuma_batch {
    int n_sys = 0;
    std::vector<spuma_ldu_t> hs;
    std::vector<SolveArgs> args;
    int threads = 256, policy = 1, grid_div = 1, grid = 0, kind = 1;
    double tuned_ms = -1.0;
    bool captured = false;
    std::vector<spuma_batch_trial> trials;   // what the tuner timed (empty: cache hit or no tuning)
    BatchTable table{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// grid: all co-resident blocks (per SM x SMs), divided by grid_div.
static spuma_status batch_configure(spuma_batch* bt, int threads, int policy, int grid_div, int num_sms)
{
    int per_sm = solve_blocks_per_sm(threads, true, bt->kind);
    if (per_sm < 1) { set_error("batch kernel cannot be resident"); return SPUMA_ERR_CUDA; }
    int grid = std::min(per_sm * num_sms, kMaxBlocks) / std::max(1, grid_div);
    if (grid < bt->n_sys) { set_error("more systems than co-resident blocks"); return SPUMA_ERR_INVALID_ARG; }
    std::vector<double> w;
    policy_weights(policy, bt->hs, w);
    bt->table.n_sys = bt->n_sys;
    if (!batch_split(bt->n_sys, w.data(), grid, bt->table.split)) { set_error("batch split failed"); return SPUMA_ERR_INVALID_ARG; }
    for (int k = 0; k < bt->n_sys; k++) bt->table.args[k] = bt->hs[k]->at<SolveArgs>(bt->hs[k]->L.args);
    bt->threads = threads;
    bt->policy = policy;
    bt->grid_div = std::max(1, grid_div);
    bt->grid = grid;
    return SPUMA_OK;
}

static spuma_status batch_launch(spuma_batch* bt, cudaStream_t s, bool count = true)
{
    for (int k = 0; k < bt->n_sys; k++) {
        spuma_ldu_t h = bt->hs[k];
        SPUMA_CUDA(cudaMemsetAsync(h->at<char>(h->L.bar), 0, h->L.status + 256 - h->L.bar, s));
    }
    spuma_status st = launch_batch_kernel(bt->table, bt->grid, bt->threads, bt->kind, s);
    if (st == SPUMA_OK && count) count_launch();
    return st;
}

static std::string batch_signature(const spuma_batch* bt, const spuma_solver_controls* ctl, int num_sms)
{
    unsigned long long hsh = 1469598103934665603ull;
    auto mix = [&](long long v) {
        hsh ^= (unsigned long long)v;
        hsh *= 1099511628211ull;
    };
    long long cells = 0;
    for (auto h : bt->hs) {
        mix(h->n);
        mix(h->nf);
        mix(h->nlev);
        cells += h->n;
    }
    char buf[256];
    snprintf(buf, sizeof buf, "sms%d-sys%d-cells%lld-pc%d-pr%d-%016llx", num_sms, bt->n_sys, cells, ctl->precond,
             ctl->precision, hsh);
    return buf;
}

static spuma_status batch_create(int32_t n_sys, const spuma_ldu_t* hs, const double* const* diag,
                                 const double* const* upper, const double* const* b, double* const* x,
                                 const spuma_solver_controls* ctl, spuma_solver_perf* perf, int32_t flags,
                                 spuma_stream_t stream, spuma_batch_t* out)
{
    if (!out) { set_error("out is NULL"); return SPUMA_ERR_INVALID_ARG; }
    *out = nullptr;
    if (n_sys < 1 || n_sys > 256 || !hs || !diag || !upper || !b || !x || !perf || !ctl_ok(ctl) ||
        (flags & ~(SPUMA_BATCH_AUTOTUNE | SPUMA_BATCH_ALLOW_DIRECT | SPUMA_BATCH_NO_GRAPH)) != 0) {
        set_error("spuma_batch_create: bad argument (1..256 systems, known flags)");
        return SPUMA_ERR_INVALID_ARG;
    }
    for (int k = 0; k < n_sys; k++) {
        if (!hs[k] || hs[k]->n < 1 || !diag[k] || !b[k] || !x[k] || (hs[k]->nf > 0 && !upper[k])) {
            set_error("spuma_batch_create: bad system " + std::to_string(k));
            return SPUMA_ERR_INVALID_ARG;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    spuma_batch* bt = new spuma_batch();
    bt->n_sys = n_sys;
    bt->kind = batch_kind(ctl->precision);
    bt->hs.assign(hs, hs + n_sys);
    bt->args.resize(n_sys);
    auto fail = [&](spuma_status st) {
        if (bt->exec) cudaGraphExecDestroy(bt->exec);
        if (bt->graph) cudaGraphDestroy(bt->graph);
        delete bt;
        return st;
    };
    for (int k = 0; k < n_sys; k++) {
        SolveArgs& a = bt->args[k];
        a = make_args(hs[k]);
        fill_controls(a, ctl);
        a.mode = MODE_SOLVE;
        a.diag_orig = diag[k];
        a.upper_orig = upper[k];
        a.b_orig = b[k];
        a.x_orig = x[k];
        a.perf = perf + k;
        a.tail_from = hs[k]->nlev;        // batch groups run every level on all their blocks
        hs[k]->prepared_precond = ctl->precond;
    }
    // trial runs of the tuner start from 0 and leave the caller's x alone
    spuma_status st;
    auto upload = [&](bool trial) -> spuma_status {
        for (int k = 0; k < n_sys; k++) {
            SolveArgs a = bt->args[k];
            if (trial) {
                a.zero_x0 = 1;
                a.no_store = 1;
            }
            SPUMA_CUDA(cudaMemcpyAsync(hs[k]->at<SolveArgs>(hs[k]->L.args), &a, sizeof(SolveArgs),
                                       cudaMemcpyHostToDevice, s));
        }
        return cudaStreamSynchronize(s) == cudaSuccess ? SPUMA_OK : cuda_fail(cudaGetLastError(), "args upload");
    };
    int num_sms = hs[0]->num_sms;
    int threads = ctl->block_threads > 0 ? ctl->block_threads : 256, policy = 1, grid_div = 1;
    if (flags & SPUMA_BATCH_AUTOTUNE) {
        if ((st = upload(true)) != SPUMA_OK) return fail(st);
        const char* path = getenv("SPUMA_TUNE_CACHE");
        std::string sig = batch_signature(bt, ctl, num_sms);
        double ms = 0;
        if (tune_cache_lookup(path, sig, &threads, &policy, &grid_div, &ms)) {
            bt->tuned_ms = ms;
        } else {
            cudaEvent_t e0, e1;
            if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
                return fail(cuda_fail(cudaGetLastError(), "cudaEventCreate"));
            // median of three timed solves (after one untimed) of a candidate;
            // a candidate that cannot run (not resident, fewer blocks than
            // systems) is skipped
            auto trial = [&](int t, int pol, int div, double* out) -> spuma_status {
                *out = -1.0;
                if (batch_configure(bt, t, pol, div, num_sms) != SPUMA_OK) return SPUMA_OK;
                spuma_status ls;
                if ((ls = batch_launch(bt, s)) != SPUMA_OK) return ls;
                float tm[3];
                for (int r = 0; r < 3; r++) {
                    cudaEventRecord(e0, s);
                    if ((ls = batch_launch(bt, s)) != SPUMA_OK) return ls;
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) return cuda_fail(cudaGetLastError(), "tune");
                    cudaEventElapsedTime(&tm[r], e0, e1);
                }
                std::sort(tm, tm + 3);
                *out = tm[1];
                bt->trials.push_back({t, pol, bt->grid_div, bt->grid, tm[1]});
                return SPUMA_OK;
            };
            // staged search: block size, then the weighting of the split,
            // then a half-size grid (fewer blocks per system: cheaper grid
            // barriers for systems too small to use them all)
            double best = 1e30;
            int bt_t = threads, bt_p = policy, bt_d = 1;
            const int cand_t[5] = {64, 128, 256, 512, 1024};
            for (int ti = 0; ti < 5; ti++) {
                double m;
                if ((st = trial(cand_t[ti], 1, 1, &m)) != SPUMA_OK) return fail(st);
                if (m >= 0.0 && m < best) { best = m; bt_t = cand_t[ti]; }
            }
            for (int pol = 0; pol < kPolicies; pol++) {
                if (pol == 1) continue;
                double m;
                if ((st = trial(bt_t, pol, 1, &m)) != SPUMA_OK) return fail(st);
                if (m >= 0.0 && m < best) { best = m; bt_p = pol; }
            }
            {
                double m;
                if ((st = trial(bt_t, bt_p, 2, &m)) != SPUMA_OK) return fail(st);
                if (m >= 0.0 && m < best) { best = m; bt_d = 2; }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (best >= 1e30) return fail((set_error("batch autotuner: no candidate could run"), SPUMA_ERR_CUDA));
            threads = bt_t;
            policy = bt_p;
            grid_div = bt_d;
            bt->tuned_ms = best;
            tune_cache_store(path, sig, threads, policy, grid_div, best);
        }
    }
    if ((st = batch_configure(bt, threads, policy, grid_div, num_sms)) != SPUMA_OK) return fail(st);
    if ((st = upload(false)) != SPUMA_OK) return fail(st);
    if (!(flags & SPUMA_BATCH_NO_GRAPH)) {
        // capture one launch (barrier resets + the persistent kernel) in a graph
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "cudaStreamCreate"));
        std::string why;
        cudaError_t eb = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (eb == cudaSuccess) {
            spuma_status ls = batch_launch(bt, cs, false);   // captured, not launched
            cudaError_t ec = cudaStreamEndCapture(cs, &bt->graph);
            cudaError_t ei = cudaErrorUnknown;
            if (ls == SPUMA_OK && ec == cudaSuccess && bt->graph)
                ei = cudaGraphInstantiate(&bt->exec, bt->graph, 0);
            if (ls == SPUMA_OK && ec == cudaSuccess && bt->graph && ei == cudaSuccess)
                bt->captured = true;
            else
                why = ls != SPUMA_OK ? std::string("launch: ") + spuma_last_error()
                      : ec != cudaSuccess ? std::string("end capture: ") + cudaGetErrorString(ec)
                                          : std::string("instantiate: ") + cudaGetErrorString(ei);
        } else {
            why = std::string("begin capture: ") + cudaGetErrorString(eb);
        }
        cudaGetLastError();
        cudaStreamDestroy(cs);
        if (!bt->captured) {
            if (bt->exec) cudaGraphExecDestroy(bt->exec);
            if (bt->graph) cudaGraphDestroy(bt->graph);
            bt->exec = nullptr;
            bt->graph = nullptr;
            if (!(flags & SPUMA_BATCH_ALLOW_DIRECT)) {
                set_error("spuma_batch_create: CUDA graph capture failed (" + why + ")");
                return fail(SPUMA_ERR_CUDA);
            }
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "batch create"));
    *out = bt;
    return SPUMA_OK;
}

extern "C" {

spuma_status spuma_batch_create(int32_t n_sys, const spuma_ldu_t* hs, const double* const* diag,
                                const double* const* upper, const double* const* b, double* const* x,
                                const spuma_solver_controls* ctl, spuma_solver_perf* perf, int32_t flags,
                                spuma_stream_t stream, spuma_batch_t* out)
{
    return host_guard("spuma_batch_create",
                      [&] { return batch_create(n_sys, hs, diag, upper, b, x, ctl, perf, flags, stream, out); });
}

spuma_status spuma_batch_run(spuma_batch_t bt, spuma_stream_t stream)
{
    if (!bt) { set_error("batch is NULL"); return SPUMA_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    if (bt->exec) {
        SPUMA_CUDA(cudaGraphLaunch(bt->exec, s));
        count_launch();
        return SPUMA_OK;
    }
    return batch_launch(bt, s);
}

spuma_status spuma_batch_info(spuma_batch_t bt, int32_t* block_threads, int32_t* grid_blocks, double* tuned_ms,
                              int32_t* graph_captured)
{
    if (!bt) { set_error("batch is NULL"); return SPUMA_ERR_INVALID_ARG; }
    if (block_threads) *block_threads = bt->threads;
    if (grid_blocks) *grid_blocks = bt->grid;
    if (tuned_ms) *tuned_ms = bt->tuned_ms;
    if (graph_captured) *graph_captured = bt->captured ? 1 : 0;
    return SPUMA_OK;
}

int32_t spuma_batch_trials(spuma_batch_t bt, int32_t max_trials, int32_t* block_threads, int32_t* split_policy,
                           int32_t* grid_blocks, double* ms)
{
    if (!bt) return 0;
    const int n = (int)bt->trials.size();
    for (int k = 0; k < n && k < max_trials; k++) {
        if (block_threads) block_threads[k] = bt->trials[k].threads;
        if (split_policy) split_policy[k] = bt->trials[k].policy;
        if (grid_blocks) grid_blocks[k] = bt->trials[k].grid;
        if (ms) ms[k] = bt->trials[k].ms;
    }
    return n;
}

spuma_status spuma_batch_destroy(spuma_batch_t bt)
{
    if (!bt) return SPUMA_OK;
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    delete bt;
    return SPUMA_OK;
}

spuma_status spuma_batch_solve(int32_t n_sys, const spuma_ldu_t* hs, const double* const* diag,
                               const double* const* upper, const double* const* b, double* const* x,
                               const spuma_solver_controls* ctl, spuma_solver_perf* perf, spuma_stream_t stream)
{
    spuma_batch_t bt = nullptr;
    spuma_status st = spuma_batch_create(n_sys, hs, diag, upper, b, x, ctl, perf, SPUMA_BATCH_NO_GRAPH, stream, &bt);
    if (st != SPUMA_OK) return st;
    st = spuma_batch_run(bt, stream);
    cudaStreamSynchronize((cudaStream_t)stream);
    spuma_batch_destroy(bt);
    return st;
}

int32_t spuma_batch_split(int32_t n_sys, const double* weights, int32_t grid, int32_t* split_out)
{
    if (!weights || !split_out) return 0;
    return batch_split(n_sys, weights, grid, split_out) ? 1 : 0;
}

int32_t spuma_tune_cache_lookup(const char* path, const char* signature, int32_t* threads, int32_t* policy,
                                int32_t* grid_div, double* ms)
{
    if (!signature || !threads || !policy || !grid_div || !ms) return 0;
    try {
        int t, p, d;
        if (!tune_cache_lookup(path, signature, &t, &p, &d, ms)) return 0;
        *threads = t;
        *policy = p;
        *grid_div = d;
        return 1;
    } catch (...) {
        return 0;   // a host failure reads as a cache miss
    }
}

int32_t spuma_tune_cache_store(const char* path, const char* signature, int32_t threads, int32_t policy,
                               int32_t grid_div, double ms)
{
    if (!signature || grid_div < 1) return 0;
    try {
        return tune_cache_store(path, signature, threads, policy, grid_div, ms) ? 1 : 0;
    } catch (...) {
        return 0;
    }
}

}  // extern "C"
