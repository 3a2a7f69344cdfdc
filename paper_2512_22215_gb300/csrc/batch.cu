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
int solve_blocks_per_sm(int threads, bool batch, int kind);
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
// A JSON object, one entry per line:  "signature": [threads, policy, ms],
static std::mutex g_tune_mu;
static std::map<std::string, std::vector<double>> g_tune_mem;

bool tune_cache_lookup(const char* path, const std::string& sig, int* threads, int* policy, double* ms)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_mem.find(sig);
    if (it == g_tune_mem.end() && path && *path) {
        FILE* f = fopen(path, "r");
        if (f) {
            char line[1024];
            while (fgets(line, sizeof line, f)) {
                char key[768];
                double t = 0, p = 0, m = 0;
                if (sscanf(line, " \"%767[^\"]\" : [ %lf , %lf , %lf ]", key, &t, &p, &m) == 4)
                    g_tune_mem[key] = {t, p, m};
            }
            fclose(f);
        }
        it = g_tune_mem.find(sig);
    }
    if (it == g_tune_mem.end()) return false;
    *threads = (int)it->second[0];
    *policy = (int)it->second[1];
    *ms = it->second[2];
    return true;
}

bool tune_cache_store(const char* path, const std::string& sig, int threads, int policy, double ms)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_mem[sig] = {(double)threads, (double)policy, ms};
    if (!path || !*path) return true;
    std::map<std::string, std::vector<double>> all;
    FILE* f = fopen(path, "r");
    if (f) {
        char line[1024];
        while (fgets(line, sizeof line, f)) {
            char key[768];
            double t = 0, p = 0, m = 0;
            if (sscanf(line, " \"%767[^\"]\" : [ %lf , %lf , %lf ]", key, &t, &p, &m) == 4) all[key] = {t, p, m};
        }
        fclose(f);
    }
    all[sig] = {(double)threads, (double)policy, ms};
    std::string tmp = std::string(path) + ".tmp";
    f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fprintf(f, "{\n");
    size_t k = 0;
    for (auto& e : all) {
        fprintf(f, "  \"%s\": [%d, %d, %.6f]%s\n", e.first.c_str(), (int)e.second[0], (int)e.second[1], e.second[2],
                ++k < all.size() ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    return std::rename(tmp.c_str(), path) == 0;
}

// Block weights per system: policy 0 = cells, 1 = cells^(4/3) (cells times
// an iteration count that grows like the mesh side).
static void policy_weights(int policy, const std::vector<spuma_ldu_t>& hs, std::vector<double>& w)
{
    w.resize(hs.size());
    for (size_t k = 0; k < hs.size(); k++) {
        double n = std::max(1, hs[k]->n);
        w[k] = policy == 0 ? n : std::pow(n, 4.0 / 3.0);
    }
}

}  // namespace spuma

using namespace spuma;

struct spuma_batch {
    int n_sys = 0;
    std::vector<spuma_ldu_t> hs;
    std::vector<SolveArgs> args;
    int threads = 256, policy = 1, grid = 0, kind = 1;
    double tuned_ms = -1.0;
    BatchTable table{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static spuma_status batch_configure(spuma_batch* bt, int threads, int policy, int num_sms)
{
    int per_sm = solve_blocks_per_sm(threads, true, bt->kind);
    if (per_sm < 1) { set_error("batch kernel cannot be resident"); return SPUMA_ERR_CUDA; }
    int grid = std::min(per_sm * num_sms, kMaxBlocks);
    if (grid < bt->n_sys) { set_error("more systems than co-resident blocks"); return SPUMA_ERR_INVALID_ARG; }
    std::vector<double> w;
    policy_weights(policy, bt->hs, w);
    bt->table.n_sys = bt->n_sys;
    if (!batch_split(bt->n_sys, w.data(), grid, bt->table.split)) { set_error("batch split failed"); return SPUMA_ERR_INVALID_ARG; }
    for (int k = 0; k < bt->n_sys; k++) bt->table.args[k] = bt->hs[k]->at<SolveArgs>(bt->hs[k]->L.args);
    bt->threads = threads;
    bt->policy = policy;
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

extern "C" {

spuma_status spuma_batch_create(int32_t n_sys, const spuma_ldu_t* hs, const double* const* diag,
                                const double* const* upper, const double* const* b, double* const* x,
                                const spuma_solver_controls* ctl, spuma_solver_perf* perf, int32_t autotune,
                                spuma_stream_t stream, spuma_batch_t* out)
{
    if (!out) { set_error("out is NULL"); return SPUMA_ERR_INVALID_ARG; }
    *out = nullptr;
    if (n_sys < 1 || n_sys > 256 || !hs || !diag || !upper || !b || !x || !perf || !ctl_ok(ctl)) {
        set_error("spuma_batch_create: bad argument (1..256 systems)");
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
    int threads = ctl->block_threads > 0 ? ctl->block_threads : 256, policy = 1;
    if (autotune) {
        if ((st = upload(true)) != SPUMA_OK) return fail(st);
        const char* path = getenv("SPUMA_TUNE_CACHE");
        std::string sig = batch_signature(bt, ctl, num_sms);
        double ms = 0;
        if (tune_cache_lookup(path, sig, &threads, &policy, &ms)) {
            bt->tuned_ms = ms;
        } else {
            cudaEvent_t e0, e1;
            if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
                return fail(cuda_fail(cudaGetLastError(), "cudaEventCreate"));
            double best = 1e30;
            int bt_t = threads, bt_p = policy;
            const int cand_t[2] = {128, 256};
            for (int ti = 0; ti < 2; ti++) {
                for (int pol = 0; pol < 2; pol++) {
                    if (batch_configure(bt, cand_t[ti], pol, num_sms) != SPUMA_OK) continue;
                    if ((st = batch_launch(bt, s)) != SPUMA_OK) return fail(st);   // warm-up
                    std::vector<float> t(3);
                    for (int r = 0; r < 3; r++) {
                        cudaEventRecord(e0, s);
                        if ((st = batch_launch(bt, s)) != SPUMA_OK) return fail(st);
                        cudaEventRecord(e1, s);
                        if (cudaEventSynchronize(e1) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "tune"));
                        cudaEventElapsedTime(&t[r], e0, e1);
                    }
                    std::sort(t.begin(), t.end());
                    if (t[1] < best) {
                        best = t[1];
                        bt_t = cand_t[ti];
                        bt_p = pol;
                    }
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            threads = bt_t;
            policy = bt_p;
            bt->tuned_ms = best;
            tune_cache_store(path, sig, threads, policy, best);
        }
    }
    if ((st = batch_configure(bt, threads, policy, num_sms)) != SPUMA_OK) return fail(st);
    if ((st = upload(false)) != SPUMA_OK) return fail(st);
    // capture one launch (barrier resets + the persistent kernel) in a graph
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "cudaStreamCreate"));
    bool captured = false;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        spuma_status ls = batch_launch(bt, cs, false);   // captured, not launched
        cudaError_t ec = cudaStreamEndCapture(cs, &bt->graph);
        if (ls == SPUMA_OK && ec == cudaSuccess && bt->graph &&
            cudaGraphInstantiate(&bt->exec, bt->graph, 0) == cudaSuccess)
            captured = true;
    }
    cudaGetLastError();
    cudaStreamDestroy(cs);
    if (!captured) {
        if (bt->exec) cudaGraphExecDestroy(bt->exec);
        if (bt->graph) cudaGraphDestroy(bt->graph);
        bt->exec = nullptr;
        bt->graph = nullptr;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "batch create"));
    *out = bt;
    return SPUMA_OK;
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

spuma_status spuma_batch_info(spuma_batch_t bt, int32_t* block_threads, int32_t* grid_blocks, double* tuned_ms)
{
    if (!bt) { set_error("batch is NULL"); return SPUMA_ERR_INVALID_ARG; }
    if (block_threads) *block_threads = bt->threads;
    if (grid_blocks) *grid_blocks = bt->grid;
    if (tuned_ms) *tuned_ms = bt->tuned_ms;
    return SPUMA_OK;
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
    spuma_status st = spuma_batch_create(n_sys, hs, diag, upper, b, x, ctl, perf, 0, stream, &bt);
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
                                double* ms)
{
    if (!signature || !threads || !policy || !ms) return 0;
    int t, p;
    if (!tune_cache_lookup(path, signature, &t, &p, ms)) return 0;
    *threads = t;
    *policy = p;
    return 1;
}

int32_t spuma_tune_cache_store(const char* path, const char* signature, int32_t threads, int32_t policy, double ms)
{
    if (!signature) return 0;
    return tune_cache_store(path, signature, threads, policy, ms) ? 1 : 0;
}

}  // extern "C"
