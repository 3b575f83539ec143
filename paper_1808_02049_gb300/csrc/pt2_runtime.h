// Host-side runtime state of libpt2, shared by pt2_api.cu (resources and the
// simple entry points) and pt2_engine.cu (planning, steps, batches, serving).
#pragma once

#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "pt2.h"
#include "pt2_internal.cuh"

namespace pt2 {

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct SystemRes {
    int n = 0;
    DevBuf h, eri, J, WS, Jx, WSx, hdx, dpair;
    int refs = 0;  // references using this system
};

struct RefRes {
    uint32_t system = 0;
    uint64_t n_det = 0;
    int na = 0, nb = 0;
    double e0 = 0.0;
    DevBuf keys, coef, hii, d0;
    DevBuf g;      // per determinant: (h_xx + p(x)) * 2^48 for the n alpha then the n beta spin-orbitals
    bool flip_symmetric = false;  // closed under alpha <-> beta exchange with equal coefficients
    int busy = 0;  // requests of the serving engine that use it
};

constexpr int kPhases = 8;

// One memory-bounded pass of an instance: the alpha-hash classes
// [c_lo, c_hi) (a set of Algorithm 2 constraints) and, for an alpha class too
// heavy for one pass, the beta-hash classes [b_lo, b_hi) within it; its terms
// and tiles.
struct Pass {
    uint32_t c_lo = 0, c_hi = 0;
    uint32_t b_lo = 0, b_hi = kNumClasses;
    uint64_t records = 0;
    uint64_t n_tiles = 0;
    bool at_most = false;  // records is an upper bound (beta classes of a heavy class in a cutoff run)
};

// One PT2 solve scheduled by the engine.
struct Job {
    RefRes *r = nullptr;
    SystemRes *s = nullptr;
    pt2_opts o{};
    uint64_t tile_target = 0;
    uint32_t cls_lo = 0, cls_hi = kNumClasses;  // alpha classes of the run (a class slice, or all)
    uint64_t pass_cap = 0;  // records one pass of this job may hold
    GenParams gp{};         // instance parameters (pass fields filled per step)
    std::vector<Pass> passes;
    uint64_t total = 0;
    size_t next = 0;        // next pass to run
    RunAcc *acc = nullptr;  // device accumulator
    // serving bookkeeping
    uint64_t ticket = 0;
    uint32_t ref_id = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    uint64_t footprint = 0;  // bytes of records its passes may hold (server admission)
    int status = PT2_ERR_BUSY;
    pt2_result result{};
};

// Device tables of one step (a set of job passes run by the same launches).
struct StepDev {
    GenParams params[kMaxBatch];
    unsigned long long det_base[kMaxBatch + 1];
    unsigned long long tile_base[kMaxBatch + 1];
    double e0[kMaxBatch];
    uint32_t iflags[kMaxBatch];  // kInst* options of each instance
    unsigned long long expected[kMaxBatch];
    RunAcc *acc[kMaxBatch];
    unsigned int n_big[kMaxBatch];
};

struct StepItem {
    Job *job;
    size_t pass;
};

struct StepPlan {
    std::vector<StepItem> items;
    uint64_t n_ctas = 0, n_tiles = 0, records = 0;
};

struct Batch;
struct Server;

}  // namespace pt2

struct pt2_ctx {
    int device = 0;
    int sm_count = 0;
    int tile_per_sm = 4, big_per_sm = 3;  // resident CTAs of the persistent kernels
    cudaStream_t stream = nullptr;
    uint64_t budget = 0, used = 0;
    std::string err;
    uint32_t next_id = 1;
    std::map<uint32_t, std::unique_ptr<pt2::SystemRes>> systems;
    std::map<uint32_t, std::unique_ptr<pt2::RefRes>> refs;
    pt2::DevBuf hash;
    // step workspace (grow-only), shared by every run, batch and the server
    pt2::DevBuf class_counts, tile_counts, tile_off, cursor, scan_tmp, recs, ref_tile, ref_count, ref_off,
        ref_cursor, ref_keys, big_list, big_max, scratch, acc, err_word, steps, gen_tab, dump_keys, dump_num,
        dump_haa, dump_count;
    pt2::DevBuf grp_counts, grp_tab;  // tile counts of a group of passes counted by one launch, and its pass tables
    uint64_t ws_gen = 0;  // bumped whenever a device buffer is reallocated
    void *steps_pinned = nullptr;  // staging of the step tables (pinned)
    size_t steps_pinned_bytes = 0;
    cudaEvent_t ev[2 * pt2::kPhases + 2] = {};
    double phase_ms[pt2::kPhases] = {};
    uint64_t launches = 0;
    // tuning table: tile target per size class (0 = default)
    uint32_t tuned_tile[8] = {};
    // serialises GPU work of pt2_run, batches and the serving engine
    std::recursive_mutex exec;
    // unfinished requests of the serving engine per reference id; its own
    // (innermost) lock, so an unload can refuse a busy reference without
    // waiting for a step that holds `exec`
    std::mutex served_mu;
    std::map<uint32_t, int> served;
    std::map<uint32_t, std::unique_ptr<pt2::Batch>> batches;
    std::unique_ptr<pt2::Server> server;
    pt2_ctx();
    ~pt2_ctx();  // defined where Batch and Server are complete
};

namespace pt2 {

int fail(pt2_ctx *c, int code, const char *fmt, ...);
int cuda_fail(pt2_ctx *c, cudaError_t e, const char *what);
int dev_alloc(pt2_ctx *c, DevBuf &b, size_t bytes, const char *what);
void dev_free(pt2_ctx *c, DevBuf &b);
int ensure(pt2_ctx *c, DevBuf &b, size_t bytes, const char *what);
SysDev sys_dev(const SystemRes &s);
uint64_t terms_per_det(int n, int na, int nb);
int status_of_err(pt2_ctx *c, uint32_t err);
GenParams gen_params(pt2_ctx *c, const SystemRes &s, const RefRes &r);
void server_stop(pt2_ctx *c);
void batches_release(pt2_ctx *c);

}  // namespace pt2

#define CK(call, what)                                              \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return pt2::cuda_fail(c, e_, what);  \
    } while (0)
