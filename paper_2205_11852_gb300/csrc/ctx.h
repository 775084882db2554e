// Private context of libtpcf, shared by the translation units of the C ABI.
#pragma once

#include <map>
#include <string>
#include <vector>

#include "plan.h"

namespace tpcf {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct PinBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// One instantiated CUDA graph of a batched tpcf_count, replayed while the
// call's plan, buffers and outputs stay the same.
struct GraphEntry {
    std::string key;
    cudaGraph_t graph = nullptr;                       // kept: its nodes address the exec's nodes
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t ev_node[2] = {nullptr, nullptr};   // event-record nodes around the pair-count kernel
    void *small = nullptr;                             // the graph's own copy of the small tables
    int kernels = 0;
    unsigned long long last_use = 0;
};

// Host-input counts run in at most this many groups of mocks, each staged
// while the previous one is counted; a group holds at least the context's
// group_kb KiB of staged positions (TPCF_OPT_HOST_GROUP_KB).
constexpr int PIPE_GROUPS_MAX = 8;

// Autotuned configuration of the batched pair count.
struct Tuned {
    int subdiv = 3;
    int chunk = 256;
    int kernel = -1;   // TPCF_KERNEL_*; -1: the context's preference
    int bps = 0;       // blocks per SM of the pair counter; 0: as many as fit
};

}  // namespace tpcf

struct tpcf_ctx {
    int device = 0;
    int n_sm = 0;
    std::string err;
    bool broken = false;
    // workspace
    std::map<std::string, tpcf::DevBuf> bufs;
    tpcf::PinBuf staging;
    cudaEvent_t staging_free = nullptr;   // recorded after the last copy out of `staging`
    bool staging_pending = false;
    int *status = nullptr;                // device status word
    unsigned long long *stats = nullptr;  // device [4]
    unsigned long long *stats_host = nullptr;  // pinned [4]
    // timing: one event pair per timed tpcf_count
    bool timing = false;
    std::vector<cudaEvent_t> ev;          // [2 * k]
    // whole-call spans of timed tpcf_count calls on their stream [2 * k], and the host-input copies [2 * k]
    std::vector<cudaEvent_t> call_ev, stage_ev;
    int n_call_timed = 0, n_stage_timed = 0;
    int n_timed = 0;
    cudaEvent_t done = nullptr;           // recorded after the stats copy of the last tpcf_count
    cudaEvent_t scratch_ev[2] = {nullptr, nullptr};   // graph event nodes point here when untimed
    int last_launches = 0;
    int last_kernels = 0;
    bool last_graph = false;
    // planner and autotuner
    int subdiv_pin = 0;
    int use_graphs = 1;
    int autotune = 1;
    std::map<std::string, tpcf::Tuned> tune_cache;
    int last_subdiv = 0, last_nc = 0, last_chunk = 0, last_blocks = 0;
    std::string device_id;                // name, SM count and compute capability (tune-cache key)
    int kernel_pref = 0;                  // TPCF_KERNEL_AUTO (the default) | _DIRECT | _GENERAL
    bool last_direct = false;             // the last tpcf_count ran the direct counter
    // split-precision Gram kernel: bound of its epilogue wait (0: built in), test-only MMA skip
    long long gram_wait_limit = 0;
    int test_skip_mma = 0;
    // test hooks read from the environment at tpcf_create: the n-th device
    // allocation of ensure() fails (TPCF_TEST_FAIL_ALLOC=n) and the n-th
    // tpcf_count fails as if a launch had failed (TPCF_TEST_FAIL_COUNT=n)
    long long fail_alloc_at = 0, n_alloc = 0;
    long long fail_count_at = 0, n_count = 0;
    // host-input counts in groups: the groups' copies run on copy_stream;
    // pipe_ev holds [0] the call's start, [1] its end (the next call's copies
    // wait for it), then per group g [2 + 2 g] copied and [3 + 2 g] counted
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> pipe_ev;
    long long group_kb = 262144;
    // graphs
    cudaStream_t cap_stream = nullptr;
    std::vector<tpcf::GraphEntry> graphs;
    unsigned long long use_clock = 0;
};

namespace tpcf {
namespace detail {

int fail(tpcf_ctx *c, int code, const std::string &msg);
int cuda_fail(tpcf_ctx *c, cudaError_t e, const char *where);
int ensure(tpcf_ctx *ctx, const char *name, size_t bytes, void **out);
int staging(tpcf_ctx *ctx, size_t bytes, void **out);
int staging_done(tpcf_ctx *ctx, cudaStream_t s);
size_t al(size_t x);
int check_ctx(tpcf_ctx *ctx);
int validate_binning(tpcf_ctx *ctx, const tpcf_binning *b);
int check_mu_width(tpcf_ctx *ctx, const tpcf_binning *b, const CountParams &p);
GramOpts gram_opts(const tpcf_ctx *ctx);
void release_graphs(tpcf_ctx *ctx);

}  // namespace detail
}  // namespace tpcf

#define CK(expr)                                                                       \
    do {                                                                               \
        cudaError_t _e = (expr);                                                       \
        if (_e != cudaSuccess) return ::tpcf::detail::cuda_fail(ctx, _e, #expr);       \
    } while (0)
