// Tensor-network contraction along a pairwise path (Sec. II-A: the
// contraction is a sequence of operations between neighbouring tensors that
// create intermediates), and the library's greedy path.
//
// Execution model.  Every step of the path is one blocked pairwise tensordot
// (gett.cu).  Steps are grouped into dependency waves (a step's wave is one
// more than the latest wave of its operands); all steps of a wave that use
// the same kernel family run in ONE grouped launch whose CTAs look up their
// problem in a device-side descriptor array.  Intermediates live in one
// device arena whose offsets are packed by lifetime (first wave written, last
// wave read).  Plans (offset tables, arena, descriptors and optionally a
// captured CUDA graph of the launches) are cached by the network's structure,
// so a later call with the same structure only patches the operand addresses
// and replays.
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <random>
#include <tuple>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "gett_common.cuh"

namespace rosnet {

void check_tensordot(rosnet_btensor A, rosnet_btensor B, int naxes, const int *axes_a,
                     const int *axes_b, int *axa, int *axb, int &rc, int64_t *shc, int64_t *blc);
int check_precision(const rosnet_opts *opts, int dtype);
int64_t reduce_ctas(const GettDesc &d);
void autotune_problem(GettDesc &d, int dtype, bool packed_ok, int reduce_mode, cudaStream_t s);
size_t tc_workspace_bytes(const GettDesc &d, int mode);
void tc_workspace_clear(const GettDesc &d, int mode, void *ws, cudaStream_t s);
void launch_tc_problem(int mode, const GettDesc &d, const GroupArgs &ga, void *ws, cudaStream_t s,
                       bool pack_a, bool pack_b, const std::function<void()> &before_gemm = {},
                       bool pdl = true);

namespace {

// offsets tables on the host (same contents as build_table_kernel)
void host_table(const ModeList &ml, int64_t total, int64_t *o0, int64_t *o1) {
    for (int64_t i = 0; i < total; ++i) {
        int64_t r = i, a = 0, b = 0;
        for (int j = ml.n - 1; j >= 0; --j) {
            int64_t d = r % ml.m[j].ext;
            r /= ml.m[j].ext;
            a += d * ml.m[j].s0;
            b += d * ml.m[j].s1;
        }
        o0[i] = a;
        o1[i] = b;
    }
}

// A global operand id: >= 0 is a step index, < 0 is leaf slot (-1 - id).
struct Step {
    int64_t ga, gb;      // operands
    int naxes;
    std::vector<int> axa, axb;
    Layout lay;          // layout of the result
    int wave;
    int last_use = -1;   // last wave that reads it
    bool forest = false; // computed in the plan's fused small-step launch (before every wave)
    int64_t table_off[3];   // M, N and K offset tables, in int64 entries
    size_t arena_off;    // SIZE_MAX: written straight into output out_net
    int out_net = -1;
    GettDesc desc;
};

struct Leaf {
    int net, t;          // first (network, tensor) holding this leaf
};

struct NetOut {
    int64_t final_gid;   // step or leaf holding network i's result before its permutation
    std::vector<int> perm;   // output axis o = result axis perm[o]
    Layout out_lay;
    bool direct = false; // the final step writes straight into the output tensor
};

struct Plan {
    int nnet = 0;
    int dtype = 0;
    int precision = 0;
    int flags = 0;
    cudaStream_t stream = nullptr;
    std::vector<Leaf> leaves;
    std::vector<Step> steps;
    std::vector<NetOut> outs;
    size_t arena_bytes = 0;
    DevBuf arena, tables, descs, partials, tcws;
    // launch list: (kind, first desc, count, total CTAs)
    struct Launch {
        int kind;
        int first;
        int count;
        int64_t tiles;
        size_t tc_ws_off;
        int64_t prog_off = 0;   // fused small steps: program, in int64 entries of `tables`
    };
    std::vector<Launch> launches;
    std::vector<int> desc_step;       // desc slot -> step index
    std::vector<GettDesc> slot_desc;  // desc slot -> static descriptor fields
    // pinned staging rings for descriptor uploads: kRing slots that hold any
    // changed range, and kSmallRing slots of kSmall descriptors for the usual
    // case of a few (a call's new output changes the final step's only), so
    // that a call uploading those waits for the copy kSmallRing calls back:
    // the host may run that far ahead of the device
    static constexpr int kRing = 4, kSmallRing = 64, kSmall = 8;
    GettDesc *pinned[kRing] = {nullptr};
    cudaEvent_t ev[kRing] = {nullptr};
    int ring = 0;
    GettDesc *pinned_small = nullptr;   // [kSmallRing][kSmall]
    cudaEvent_t ev_small[kSmallRing] = {nullptr};
    int ring_small = 0;
    cudaGraphExec_t graph = nullptr;
    cudaGraph_t graph_src = nullptr;           // kept for event-node updates
    // graphs cannot be captured on the legacy default stream: a plan called
    // there replays its graph on a stream of its own, ordered after and
    // before the caller's work by two events
    cudaStream_t side = nullptr;
    cudaEvent_t join[2] = {nullptr, nullptr};
    cudaGraphNode_t ev_node[3] = {nullptr, nullptr, nullptr};
    int graph_nodes = 0;
    std::vector<GettDesc> mirror;              // descriptor contents last enqueued
    bool mirror_valid = false;
    // timing of the heaviest launch (ROSNET_OPT_TIMING)
    int heavy = -1;
    double heavy_flops = 0, heavy_bytes = 0;
    int heavy_kind = -1;
    static constexpr int kTimingRing = 4096;
    // 3 * kTimingRing, created lazily: per slot the heaviest launch's start
    // (before its operand packs), its GEMM kernel's start, and its end
    std::vector<cudaEvent_t> tev;
    int tpos = 0;
    int64_t steps_requested = 0;               // path steps before common steps were merged
    uint64_t last_used = 0;                    // cache clock of the latest call
    // pinned-host spill: while spilled the offset tables (the one part of the
    // device state that is not scratch or rebuilt per call) live in
    // page-locked host memory and every device buffer and the graph are
    // released; the device addresses they had are kept to re-point the
    // descriptors when the plan is restored
    bool spilled = false;
    void *host_tables = nullptr;
    const char *old_tables = nullptr, *old_partials = nullptr;
    ~Plan() {
        // device buffers go first, while every stream they were allocated or
        // last used on still exists (the side stream is destroyed below)
        if (side) cudaStreamSynchronize(side);
        arena.reset();
        tables.reset();
        descs.reset();
        partials.reset();
        tcws.reset();
        for (int i = 0; i < kRing; ++i) {
            if (ev[i]) { cudaEventSynchronize(ev[i]); cudaEventDestroy(ev[i]); }
            if (pinned[i]) cudaFreeHost(pinned[i]);
        }
        for (cudaEvent_t &e : ev_small)
            if (e) { cudaEventSynchronize(e); cudaEventDestroy(e); }
        if (pinned_small) cudaFreeHost(pinned_small);
        if (graph) cudaGraphExecDestroy(graph);
        if (graph_src) cudaGraphDestroy(graph_src);
        if (host_tables) cudaFreeHost(host_tables);
        if (side) { cudaStreamSynchronize(side); cudaStreamDestroy(side); }
        for (cudaEvent_t e : join) if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : tev) if (e) cudaEventDestroy(e);
    }
};

// A layout of `cur`'s shape whose storage order is `order` (logical axes,
// outermost first): block-major over the axes in that order, each axis either
// a whole grid axis or wholly inside the block, the slowest axes in `order`
// made grid axes until a block holds at most maxblk entries (maxblk <= 0: one
// block).  Element x then sits at the row-major position of x's coordinates
// taken in `order`.
Layout ordered_layout(const Layout &cur, const std::vector<int> &order, int64_t maxblk) {
    const int r = cur.rank;
    int64_t sh[kMaxRank], bl[kMaxRank];
    int64_t bs = 1;
    for (int j = 0; j < r; ++j) {
        sh[j] = cur.shape[order[j]];
        bl[j] = sh[j];
        bs *= sh[j];
    }
    for (int j = 0; j < r && maxblk > 0 && bs > maxblk; ++j) {
        bs /= sh[j] > 0 ? sh[j] : 1;
        bl[j] = 1;
    }
    Layout P;
    P.init(r, sh, bl);
    Layout L = P;
    for (int j = 0; j < r; ++j) {
        const int x = order[j];
        L.shape[x] = P.shape[j];
        L.block[x] = P.block[j];
        L.gstride[x] = P.gstride[j];
        L.lstride[x] = P.lstride[j];
    }
    return L;
}

// Cached plans.  Deliberately never destroyed at process exit: by then the
// CUDA runtime or an injected allocator (e.g. one implemented in Python) may
// already be gone.  rosnet_release_plans() frees them explicitly.
std::mutex g_plan_mu;
// Plans are looked up by a 128-bit hash of everything the plan depends on.
struct Key128 {
    uint64_t a = 0x9E3779B97F4A7C15ull, b = 0xC2B2AE3D27D4EB4Full;
    void put(int64_t v) {
        uint64_t x = (uint64_t)v;
        a ^= x + 0x9E3779B97F4A7C15ull + (a << 6) + (a >> 2);
        a *= 0xBF58476D1CE4E5B9ull;
        b = (b ^ (x * 0x94D049BB133111EBull)) * 0xD6E8FEB86659FD93ull;
        b ^= b >> 31;
    }
    bool operator==(const Key128 &o) const { return a == o.a && b == o.b; }
};
struct Key128Hash {
    size_t operator()(const Key128 &k) const { return (size_t)(k.a ^ (k.b * 31)); }
};
auto &g_plans = *new std::unordered_map<Key128, std::unique_ptr<Plan>, Key128Hash>();
// (plan, ring slot) of every timed launch not yet drained
auto &g_timing_log = *new std::vector<std::pair<Plan *, int>>();
// at most this many cached plans (0: no limit); the least recently used go first
int32_t g_plan_limit = 0;
uint64_t g_plan_clock = 0;

// Free least recently used plans until at most n remain (g_plan_mu held).
// Work a freed plan already enqueued completes normally: its buffers are
// released in stream order and a graph still running is freed on completion.
void evict_plans_to(size_t n) {
    while (g_plans.size() > n) {
        auto victim = g_plans.begin();
        for (auto it = g_plans.begin(); it != g_plans.end(); ++it)
            if (it->second->last_used < victim->second->last_used) victim = it;
        Plan *vp = victim->second.get();
        g_timing_log.erase(std::remove_if(g_timing_log.begin(), g_timing_log.end(),
                                          [vp](const std::pair<Plan *, int> &e) { return e.first == vp; }),
                           g_timing_log.end());
        g_plans.erase(victim);
    }
}

// Leaf slots shared by equal tensors (same storage and layout) across the
// networks of a call; slot[i][t] for tensor t of network i.  Tensors are
// grouped by storage pointer in an open-addressing table (reused between
// calls, no allocation in steady state); within a group the layouts decide.
static bool same_tensor_view(rosnet_btensor x, rosnet_btensor y) {
    if (y->pstride != x->pstride || y->dtype != x->dtype || y->lay.rank != x->lay.rank) return false;
    for (int a = 0; a < x->lay.rank; ++a)
        if (y->lay.shape[a] != x->lay.shape[a] || y->lay.gstride[a] != x->lay.gstride[a] ||
            y->lay.lstride[a] != x->lay.lstride[a] || y->lay.block[a] != x->lay.block[a])
            return false;
    return true;
}

std::vector<std::vector<int>> leaf_slots(int nnet, const rosnet_network *nets, std::vector<Leaf> *leaves) {
    struct Ent { const void *p; int rep; int next; };   // next: same storage, other layout
    thread_local std::vector<int> head;
    thread_local std::vector<Ent> ents;
    thread_local std::vector<rosnet_btensor> rep;
    size_t total = 0;
    for (int i = 0; i < nnet; ++i) total += (size_t)std::max(nets[i].ntensors, 0);
    size_t cap = 16;
    while (cap < 2 * total) cap <<= 1;
    head.assign(cap, -1);
    ents.clear();
    rep.clear();
    std::vector<std::vector<int>> slot(nnet);
    for (int i = 0; i < nnet; ++i) {
        slot[i].resize(nets[i].ntensors);
        for (int t = 0; t < nets[i].ntensors; ++t) {
            rosnet_btensor x = nets[i].tensors[t];
            uint64_t hv = (uint64_t)(uintptr_t)x->data * 0x9E3779B97F4A7C15ull;
            size_t h = (size_t)(hv >> 32) & (cap - 1);
            while (head[h] >= 0 && ents[head[h]].p != x->data) h = (h + 1) & (cap - 1);
            int found = -1, last = -1;
            for (int e = head[h]; e >= 0; e = ents[e].next) {
                if (same_tensor_view(x, rep[ents[e].rep])) { found = ents[e].rep; break; }
                last = e;
            }
            if (found < 0) {
                found = (int)rep.size();
                rep.push_back(x);
                ents.push_back({x->data, found, -1});
                const int e = (int)ents.size() - 1;
                if (last >= 0) ents[last].next = e;
                else head[h] = e;
                if (leaves) leaves->push_back({i, t});
            }
            slot[i][t] = found;
        }
    }
    return slot;
}

Key128 plan_key(int nnet, const rosnet_network *nets, const rosnet_path *paths,
                const std::vector<std::vector<int>> &slot, int prec, int flags, int64_t maxblk,
                cudaStream_t s) {
    Key128 k;
    k.put(nnet);
    k.put(prec);
    k.put(flags);
    k.put(maxblk);
    k.put((int64_t)(intptr_t)s);
    for (int i = 0; i < nnet; ++i) {
        const rosnet_network *net = &nets[i];
        k.put(net->ntensors);
        for (int t = 0; t < net->ntensors; ++t) {
            rosnet_btensor x = net->tensors[t];
            k.put(slot[i][t]);
            k.put(x->dtype);
            k.put(x->lay.rank);
            for (int a = 0; a < x->lay.rank; ++a) {
                k.put(x->lay.shape[a]);
                k.put(x->lay.block[a]);
                k.put(x->lay.gstride[a]);
                k.put(x->lay.lstride[a]);
                k.put(net->labels[t][a]);
            }
        }
        k.put(net->nout);
        for (int o = 0; o < net->nout; ++o) k.put(net->out_labels[o]);
        k.put(paths[i].nsteps);
        for (int j = 0; j < 2 * paths[i].nsteps; ++j) k.put(paths[i].pairs[j]);
    }
    return k;
}

void validate_network(const rosnet_network *net) {
    if (!net || net->ntensors < 1 || !net->tensors || !net->ranks || !net->labels)
        RN_FAIL(ROSNET_ERR_INVALID_ARG, "malformed network");
    if (net->nout < 0 || (net->nout > 0 && !net->out_labels))
        RN_FAIL(ROSNET_ERR_INVALID_ARG, "malformed output labels");
    if (net->nout > kMaxRank) RN_FAIL(ROSNET_ERR_RANK_LIMIT, "output rank > 64");
    std::unordered_map<int64_t, int> count;
    int dtype = 0;
    for (int t = 0; t < net->ntensors; ++t) {
        rosnet_btensor x = net->tensors[t];
        if (!x) RN_FAIL(ROSNET_ERR_INVALID_ARG, "NULL tensor in network");
        if (net->ranks[t] != x->lay.rank) RN_FAIL(ROSNET_ERR_INVALID_ARG, "rank does not match tensor");
        if (x->lay.rank > 0 && !net->labels[t]) RN_FAIL(ROSNET_ERR_INVALID_ARG, "NULL labels");
        if (t == 0) dtype = x->dtype;
        else if (x->dtype != dtype) RN_FAIL(ROSNET_ERR_DTYPE, "network tensors differ in dtype");
        for (int i = 0; i < x->lay.rank; ++i) {
            for (int j = 0; j < i; ++j)
                if (net->labels[t][j] == net->labels[t][i])
                    RN_FAIL(ROSNET_ERR_UNSUPPORTED, "a label repeated on one tensor (trace)");
            count[net->labels[t][i]]++;
        }
    }
    std::unordered_map<int64_t, int> outc;
    for (int i = 0; i < net->nout; ++i) {
        if (outc[net->out_labels[i]]++) RN_FAIL(ROSNET_ERR_INVALID_ARG, "repeated output label");
        if (count[net->out_labels[i]] != 1)
            RN_FAIL(ROSNET_ERR_INVALID_ARG, "an output label must be carried by exactly one tensor");
    }
    for (auto &kv : count) {
        if (kv.second > 2) RN_FAIL(ROSNET_ERR_UNSUPPORTED, "a label carried by more than two tensors");
        if (kv.second == 1 && !outc.count(kv.first))
            RN_FAIL(ROSNET_ERR_INVALID_ARG, "an open label is missing from out_labels");
    }
}

std::unique_ptr<Plan> build_plan(int nnet, const rosnet_network *nets, const rosnet_path *paths,
                                 const std::vector<std::vector<int>> &slot, std::vector<Leaf> leaves,
                                 int prec, int flags, int64_t maxblk, cudaStream_t s) {
    auto plan = std::make_unique<Plan>();
    plan->nnet = nnet;
    plan->dtype = nets[0].tensors[0]->dtype;
    plan->precision = prec;
    plan->flags = flags;
    plan->stream = s;
    plan->leaves = std::move(leaves);
    plan->outs.resize(nnet);
    std::unordered_map<std::string, int64_t> seen;   // step signature -> step index
    auto lay_of = [&](int64_t g) -> const Layout & {
        if (g >= 0) return plan->steps[g].lay;
        const Leaf &L = plan->leaves[-1 - g];
        return nets[L.net].tensors[L.t]->lay;
    };
    auto wave_of = [&](int64_t g) { return g >= 0 ? plan->steps[g].wave : 0; };
    for (int i = 0; i < nnet; ++i) {
        const rosnet_network *net = &nets[i];
        const rosnet_path *path = &paths[i];
        if (net->tensors[0]->dtype != plan->dtype) RN_FAIL(ROSNET_ERR_DTYPE, "networks differ in dtype");
        const int nt = net->ntensors;
        if (path->nsteps != nt - 1 || (path->nsteps > 0 && !path->pairs))
            RN_FAIL(ROSNET_ERR_INVALID_ARG, "a path must have ntensors - 1 steps");
        plan->steps_requested += path->nsteps;
        const int nid = nt + path->nsteps;
        std::vector<std::vector<int64_t>> labels(nid);
        std::vector<int64_t> gid(nid);
        std::vector<int> alive(nid, 0);
        for (int t = 0; t < nt; ++t) {
            labels[t].assign(net->labels[t], net->labels[t] + net->ranks[t]);
            gid[t] = -1 - slot[i][t];
            alive[t] = 1;
        }
        for (int st = 0; st < path->nsteps; ++st) {
            const int li = path->pairs[2 * st], lj = path->pairs[2 * st + 1];
            if (li < 0 || lj < 0 || li >= nt + st || lj >= nt + st || li == lj || !alive[li] || !alive[lj])
                RN_FAIL(ROSNET_ERR_INVALID_ARG, "path step " + std::to_string(st) + " uses a dead or unknown id");
            alive[li] = alive[lj] = 0;
            const int64_t ga = gid[li], gb = gid[lj];
            const Layout &la = lay_of(ga), &lb = lay_of(gb);
            std::vector<int> axa, axb;
            std::vector<int64_t> lc, shc, blc;
            std::vector<bool> ca(la.rank, false), cb(lb.rank, false);
            for (int x = 0; x < la.rank; ++x)
                for (int y = 0; y < lb.rank; ++y)
                    if (labels[li][x] == labels[lj][y]) {
                        if (la.shape[x] != lb.shape[y])
                            RN_FAIL(ROSNET_ERR_SHAPE, "a bond has different extents on its two tensors");
                        axa.push_back(x);
                        axb.push_back(y);
                        ca[x] = cb[y] = true;
                    }
            for (int x = 0; x < la.rank; ++x)
                if (!ca[x]) { lc.push_back(labels[li][x]); shc.push_back(la.shape[x]); blc.push_back(la.block[x]); }
            for (int y = 0; y < lb.rank; ++y)
                if (!cb[y]) { lc.push_back(labels[lj][y]); shc.push_back(lb.shape[y]); blc.push_back(lb.block[y]); }
            if ((int)lc.size() > kMaxRank) RN_FAIL(ROSNET_ERR_RANK_LIMIT, "intermediate rank > 64");
            if (maxblk > 0) {
                int64_t bs = 1;
                for (int64_t b : blc) bs *= b;
                for (size_t x = 0; x < blc.size() && bs > maxblk; ++x) {
                    bs /= blc[x];
                    blc[x] = 1;
                }
            }
            // the same operands contracted the same way give the same tensor:
            // compute it once (slices share every step that no sliced bond reaches)
            std::string sig;
            auto put = [&sig](int64_t v) { sig.append((const char *)&v, sizeof(v)); };
            put(ga);
            put(gb);
            put((int64_t)axa.size());
            for (size_t x = 0; x < axa.size(); ++x) { put(axa[x]); put(axb[x]); }
            for (size_t x = 0; x < blc.size(); ++x) put(blc[x]);
            auto it = seen.find(sig);
            int64_t g;
            if (it != seen.end()) {
                g = it->second;
            } else {
                Step S;
                S.ga = ga;
                S.gb = gb;
                S.naxes = (int)axa.size();
                S.axa = axa;
                S.axb = axb;
                S.lay.init((int)lc.size(), shc.data(), blc.data());
                S.wave = std::max(wave_of(ga), wave_of(gb)) + 1;
                S.arena_off = 0;
                g = (int64_t)plan->steps.size();
                plan->steps.push_back(std::move(S));
                seen.emplace(std::move(sig), g);
                for (int64_t op : {ga, gb})   // leaves live for the whole call
                    if (op >= 0) plan->steps[op].last_use = std::max(plan->steps[op].last_use, plan->steps[g].wave);
            }
            const int id = nt + st;
            gid[id] = g;
            labels[id] = lc;
            alive[id] = 1;
        }
        // result of network i and its output permutation
        const int last = path->nsteps > 0 ? nt + path->nsteps - 1 : 0;
        const std::vector<int64_t> &fl = labels[last];
        if ((int)fl.size() != net->nout)
            RN_FAIL(ROSNET_ERR_INVALID_ARG, "path leaves labels open that are not outputs");
        NetOut &O = plan->outs[i];
        O.final_gid = gid[last];
        O.perm.resize(net->nout);
        bool ident = true;
        for (int o = 0; o < net->nout; ++o) {
            int pos = -1;
            for (int x = 0; x < (int)fl.size(); ++x)
                if (fl[x] == net->out_labels[o]) pos = x;
            if (pos < 0) RN_FAIL(ROSNET_ERR_INVALID_ARG, "output label not produced by the path");
            O.perm[o] = pos;
            if (pos != o) ident = false;
        }
        const Layout &fin = lay_of(O.final_gid);
        std::vector<int64_t> osh(net->nout), obl(net->nout);
        for (int o = 0; o < net->nout; ++o) {
            osh[o] = fin.shape[O.perm[o]];
            obl[o] = fin.block[O.perm[o]];
        }
        O.out_lay.init(net->nout, osh.data(), obl.data());
        O.direct = ident && O.final_gid >= 0;
    }
    // a final step writes straight into its output unless another network's
    // output or a later step also needs it
    const int end_wave = 1 << 30;
    for (int i = 0; i < nnet; ++i) {
        NetOut &O = plan->outs[i];
        if (O.final_gid < 0) continue;
        Step &S = plan->steps[O.final_gid];
        if (O.direct && S.out_net < 0 && S.last_use < 0) {
            S.out_net = i;
            S.arena_off = SIZE_MAX;
        } else {
            O.direct = false;
            S.last_use = end_wave;   // copied into the output after the last wave
        }
    }
    // Storage order of the intermediates read by the packed FP32 kernel.  That
    // kernel loads its tiles of an operand viewed as a dense K x rows matrix
    // straight from memory with TMA; an intermediate stored with its
    // contracted axes outermost (in the order of the other operand's) and its
    // free axes innermost is such a matrix, so no pack pass runs for it.  The
    // step that produces it writes that order through its output offset
    // tables at no cost: the permutation of a block pair (Sec. II-C step 3) is
    // folded into the producer's stores and the consumer's tensor map.  An
    // intermediate takes the order of its first packed consumer; its blocks
    // become the innermost axes in that order (the slowest ones turned into
    // grid axes until a block holds at most max_block_entries).
    if (plan->dtype == ROSNET_C64) {
        const int red0 = (flags & ROSNET_OPT_REDUCE_SEQUENTIAL) ? kReduceSequential
                         : (flags & ROSNET_OPT_REDUCE_TREE) ? kReduceTree
                         : (flags & ROSNET_OPT_REDUCE_COMMUTATIVE) ? kReduceCommutative : kReduceAuto;
        std::vector<char> laid(plan->steps.size(), 0);
        auto axis_stride = [](const Layout &L, int x) { return L.block[x] == 1 ? L.gstride[x] : L.lstride[x]; };
        for (size_t g = 0; g < plan->steps.size(); ++g) {
            const Step &S = plan->steps[g];
            const Layout &la = lay_of(S.ga), &lb = lay_of(S.gb);
            int64_t K = 1;
            for (int i = 0; i < S.naxes; ++i) K *= la.shape[S.axa[i]];
            if (K == 0 || la.numel == 0 || lb.numel == 0) continue;
            GettDesc t;
            memset(&t, 0, sizeof(t));
            t.M = la.numel / K;
            t.N = lb.numel / K;
            t.K = K;
            // intermediates will be laid out dense for this consumer (leaves never are)
            t.flags = (S.ga >= 0 ? kFlagADense : 0) | (S.gb >= 0 ? kFlagBDense : 0);
            choose_kernel(t, plan->dtype, prec, red0);
            if (t.kind != kKindPackF32) continue;
            // order of the contracted pairs: as given, or a leaf operand's own
            // (outermost first), which the intermediate side then follows
            std::vector<int> pairs(S.naxes);
            for (int i = 0; i < S.naxes; ++i) pairs[i] = i;
            if ((S.ga < 0) != (S.gb < 0)) {
                const Layout &leaf = S.ga < 0 ? la : lb;
                const std::vector<int> &ax = S.ga < 0 ? S.axa : S.axb;
                std::stable_sort(pairs.begin(), pairs.end(), [&](int i, int j) {
                    return axis_stride(leaf, ax[i]) > axis_stride(leaf, ax[j]);
                });
            }
            for (int side = 0; side < 2; ++side) {
                const int64_t op = side ? S.gb : S.ga;
                if (op < 0 || laid[op] || plan->steps[op].arena_off == SIZE_MAX) continue;
                const std::vector<int> &ax = side ? S.axb : S.axa;
                Layout &L = plan->steps[op].lay;
                std::vector<char> contracted(L.rank, 0);
                std::vector<int> order;
                for (int i : pairs) {
                    order.push_back(ax[i]);
                    contracted[ax[i]] = 1;
                }
                for (int x = 0; x < L.rank; ++x)
                    if (!contracted[x]) order.push_back(x);
                L = ordered_layout(L, order, maxblk);
                laid[op] = 1;
            }
        }
    }
    // the GEMM view of every step, and the fused small steps: a step whose
    // kernel would be gett_small_kernel, with at most kForestMacs complex
    // multiply-adds, and whose operands are leaves or other such steps is
    // eligible; when the first W waves hold eligible steps only, those steps
    // are computed in one launch ahead of every other (gett_forest_kernel),
    // which replaces W launches by one of at most W dependent levels.  The
    // groups they form (connected through producer -> consumer) go one per
    // CTA; a group above kForestGroupMacs in total or kForestMaxSteps steps
    // stays in the waves
    const int red = (flags & ROSNET_OPT_REDUCE_SEQUENTIAL) ? kReduceSequential
                    : (flags & ROSNET_OPT_REDUCE_TREE) ? kReduceTree
                    : (flags & ROSNET_OPT_REDUCE_COMMUTATIVE) ? kReduceCommutative : kReduceAuto;
    std::vector<GettView> views(plan->steps.size());
    for (size_t g = 0; g < plan->steps.size(); ++g) {
        Step &S = plan->steps[g];
        views[g] = make_view(lay_of(S.ga), lay_of(S.gb), S.lay, S.naxes, S.axa.data(), S.axb.data());
    }
    // kernel of step g as the descriptor pass below chooses it (table
    // addresses do not enter the choice; the autotuner never changes a small step)
    auto chosen_kind = [&](size_t g) {
        const Step &S = plan->steps[g];
        GettDesc t;
        memset(&t, 0, sizeof(t));
        fill_desc_tables(t, views[g], nullptr, nullptr, nullptr);
        if (S.ga < 0) t.flags &= ~kFlagADense;
        if (S.gb < 0) t.flags &= ~kFlagBDense;
        choose_kernel(t, plan->dtype, prec, red);
        return std::make_tuple(t.kind, (double)t.M * (double)t.N * (double)t.K, t.M * t.N);
    };
    std::vector<int> comp(plan->steps.size(), -1);   // fused group of each fused step (its root's index)
    if (!(flags & ROSNET_OPT_NOGROUP)) {
        constexpr double kForestMacs = 65536.0, kForestGroupMacs = 262144.0;
        constexpr int64_t kForestEntries = kForestThreads / 2;   // a level's entries stay about one per thread
        std::vector<double> macs(plan->steps.size(), 0.0);
        int wmax = 1 << 30;   // the first waves that hold eligible steps only
        for (size_t g = 0; g < plan->steps.size(); ++g) {   // producers come before their consumers
            Step &S = plan->steps[g];
            const auto km = chosen_kind(g);
            S.forest = std::get<0>(km) == kKindSmall && std::get<1>(km) > 0 && std::get<1>(km) <= kForestMacs &&
                       std::get<2>(km) <= kForestEntries && (S.ga < 0 || plan->steps[S.ga].forest) &&
                       (S.gb < 0 || plan->steps[S.gb].forest);
            macs[g] = std::get<1>(km);
            if (!S.forest) wmax = std::min(wmax, S.wave - 1);
        }
        for (Step &S : plan->steps) S.forest = S.forest && S.wave <= wmax;
        // groups: union-find over producer -> consumer edges between fused steps
        std::vector<int> up(plan->steps.size());
        for (size_t g = 0; g < up.size(); ++g) up[g] = (int)g;
        auto find = [&](int x) {   // root of x's group, with path halving (no recursion)
            while (up[x] != x) {
                up[x] = up[up[x]];
                x = up[x];
            }
            return x;
        };
        for (size_t g = 0; g < plan->steps.size(); ++g) {
            const Step &S = plan->steps[g];
            if (!S.forest) continue;
            for (int64_t op : {S.ga, S.gb})
                if (op >= 0 && plan->steps[op].forest) up[find((int)op)] = find((int)g);
        }
        std::unordered_map<int, double> gmacs;
        std::unordered_map<int, int> gsteps;
        for (size_t g = 0; g < plan->steps.size(); ++g)
            if (plan->steps[g].forest) {
                gmacs[find((int)g)] += macs[g];
                ++gsteps[find((int)g)];
            }
        for (size_t g = 0; g < plan->steps.size(); ++g) {
            Step &S = plan->steps[g];
            if (!S.forest) continue;
            const int r = find((int)g);
            if (gmacs[r] > kForestGroupMacs || gsteps[r] > kForestMaxSteps) S.forest = false;
            else comp[g] = r;
        }
    }
    // arena: every step not written straight into an output, packed by
    // lifetime with a sweep over the waves: a step's bytes are reserved from
    // the wave that writes it to the last wave that reads it, then returned to
    // a first-fit free list (coalescing neighbours).  Fused small steps run
    // before every wave, concurrently in their groups: they are written at
    // wave 0, so no two of them share bytes
    {
        const size_t el2 = 2 * (plan->dtype == ROSNET_C64 ? 4 : 8);
        std::vector<int> order;
        for (size_t g = 0; g < plan->steps.size(); ++g)
            if (plan->steps[g].arena_off != SIZE_MAX) order.push_back((int)g);
        auto written = [&](int x) { return plan->steps[x].forest ? 0 : plan->steps[x].wave; };
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return written(x) < written(y); });
        std::map<size_t, size_t> freel;                       // offset -> size
        std::multimap<int, std::pair<size_t, size_t>> ends;   // release wave -> (off, size)
        size_t top = 0;
        auto release = [&](size_t off, size_t sz) {
            auto it = freel.emplace(off, sz).first;
            auto nx = std::next(it);
            if (nx != freel.end() && it->first + it->second == nx->first) {
                it->second += nx->second;
                freel.erase(nx);
            }
            if (it != freel.begin()) {
                auto pv = std::prev(it);
                if (pv->first + pv->second == it->first) {
                    pv->second += it->second;
                    freel.erase(it);
                }
            }
        };
        for (int g : order) {
            Step &S = plan->steps[g];
            while (!ends.empty() && ends.begin()->first < written(g)) {   // free slots dead before this wave
                release(ends.begin()->second.first, ends.begin()->second.second);
                ends.erase(ends.begin());
            }
            size_t bytes = ((size_t)S.lay.numel * el2 + 255) & ~(size_t)255;
            if (bytes == 0) bytes = 256;
            size_t off = SIZE_MAX;
            for (auto it = freel.begin(); it != freel.end(); ++it)
                if (it->second >= bytes) {
                    off = it->first;
                    const size_t rest = it->second - bytes;
                    freel.erase(it);
                    if (rest) freel.emplace(off + bytes, rest);
                    break;
                }
            if (off == SIZE_MAX) {
                off = top;
                top += bytes;
            }
            S.arena_off = off;
            const int to = S.last_use < 0 ? std::max(S.wave, 0) : S.last_use;
            ends.emplace(to, std::make_pair(off, bytes));
        }
        plan->arena_bytes = top;
    }
    // offset tables (host-built, one upload).  A table depends only on the
    // digits of its index class (extents and strides in both tensors), so
    // classes with equal digits -- the same step in every slice of a network,
    // repeated gate contractions -- share one copy.
    static_assert(sizeof(Mode) == 3 * sizeof(int64_t), "a digit list is compared as bytes");
    // The large class of a low-arithmetic-intensity step (gate kernel) is
    // kept as a mode record instead of a table as large as the tensor.
    std::unordered_map<std::string, int64_t> table_at;   // digits -> first entry
    std::vector<std::tuple<size_t, int, bool>> owners;   // (step, class, record) that fills each table
    int64_t tab_entries = 0;
    auto class_of = [&](const GettView &v, int c) -> std::pair<const ModeList *, int64_t> {
        return c == 0 ? std::make_pair(&v.M, v.Mtot) : c == 1 ? std::make_pair(&v.N, v.Ntot)
                                                               : std::make_pair(&v.K, v.Ktot);
    };
    for (size_t g = 0; g < plan->steps.size(); ++g) {
        Step &S = plan->steps[g];
        const int rec = gate_record_class(views[g], plan->dtype, prec, red,
                                          (S.ga < 0 ? kFlagADense : 0) | (S.gb < 0 ? kFlagBDense : 0));
        for (int c = 0; c < 3; ++c) {
            const auto mt = class_of(views[g], c);
            const bool is_rec = c == rec;
            std::string key(is_rec ? "R" : "T");
            key.append((const char *)&mt.second, sizeof(int64_t));
            key.append((const char *)mt.first->m, (size_t)mt.first->n * sizeof(Mode));
            auto ins = table_at.emplace(std::move(key), tab_entries);
            if (ins.second) {
                owners.emplace_back(g, c, is_rec);
                tab_entries += is_rec ? record_entries(*mt.first) : 2 * mt.second;
            }
            S.table_off[c] = ins.first->second;
        }
    }
    // the fused launch's program: its steps ordered by (group, level, index),
    // a step's level one more than its fused producers' (0 on leaves); per
    // group its run of levels, per level its run of descriptors
    std::vector<int> forest_order;
    std::vector<int64_t> prog;
    {
        std::vector<int> level(plan->steps.size(), 0);
        for (size_t g = 0; g < plan->steps.size(); ++g) {
            const Step &S = plan->steps[g];
            if (!S.forest) continue;
            for (int64_t op : {S.ga, S.gb})
                if (op >= 0 && plan->steps[op].forest) level[g] = std::max(level[g], level[op] + 1);
            forest_order.push_back((int)g);
        }
        std::stable_sort(forest_order.begin(), forest_order.end(), [&](int x, int y) {
            return comp[x] != comp[y] ? comp[x] < comp[y] : level[x] < level[y];
        });
        std::vector<int64_t> cta_groups, groups;   // groups: (first, count) pairs
        for (size_t i = 0; i < forest_order.size(); ++i) {
            const int g = forest_order[i];
            const bool new_cta = i == 0 || comp[forest_order[i - 1]] != comp[g];
            if (new_cta) cta_groups.push_back((int64_t)groups.size() / 2);
            if (new_cta || level[forest_order[i - 1]] != level[g]) {
                groups.push_back((int64_t)i);
                groups.push_back(0);
            }
            ++groups.back();
        }
        if (!forest_order.empty()) {
            const int64_t ncta = (int64_t)cta_groups.size();
            cta_groups.push_back((int64_t)groups.size() / 2);
            prog.push_back(ncta);
            prog.insert(prog.end(), cta_groups.begin(), cta_groups.end());
            prog.insert(prog.end(), groups.begin(), groups.end());
        }
    }
    const int64_t prog_off = tab_entries;
    tab_entries += (int64_t)prog.size();
    std::vector<int64_t> htab(std::max<int64_t>(tab_entries, 1));
    std::copy(prog.begin(), prog.end(), htab.begin() + prog_off);
    for (const auto &o : owners) {
        const auto mt = class_of(views[std::get<0>(o)], std::get<1>(o));
        int64_t *t = htab.data() + plan->steps[std::get<0>(o)].table_off[std::get<1>(o)];
        if (std::get<2>(o)) host_mode_record(*mt.first, t);
        else host_table(*mt.first, mt.second, t, t + mt.second);
    }
    plan->tables = DevBuf(htab.size() * sizeof(int64_t), s);
    plan->arena = DevBuf(std::max<size_t>(plan->arena_bytes, 256), s);
    RN_CHECK_CUDA(cudaMemcpyAsync(plan->tables.p, htab.data(), htab.size() * sizeof(int64_t),
                                  cudaMemcpyHostToDevice, s));
    // descriptors, grouped by (wave, kind); split-K problems of a wave get a
    // reduction launch right after their wave's launches
    const int64_t *dtab = (const int64_t *)plan->tables.p;
    std::map<std::pair<int, int>, std::vector<int>> groups;
    std::map<int, std::vector<int>> split_of_wave, atomic_of_wave;
    for (size_t g = 0; g < plan->steps.size(); ++g) {
        Step &S = plan->steps[g];
        const int st = (int)g;
        memset(&S.desc, 0, sizeof(S.desc));
        fill_desc_tables(S.desc, views[g], dtab + S.table_off[0], dtab + S.table_off[1],
                         dtab + S.table_off[2]);
        // leaves change address from call to call: never read in place by a
        // tensor map that a captured graph would keep
        if (S.ga < 0) S.desc.flags &= ~kFlagADense;
        if (S.gb < 0) S.desc.flags &= ~kFlagBDense;
        choose_kernel(S.desc, plan->dtype, prec, red);
        if (S.desc.M * S.desc.N == 0) continue;  // empty result: nothing to launch
        if (S.forest) {   // computed in the fused launch
            if (S.desc.kind != kKindSmall) RN_FAIL(ROSNET_ERR_CUDA, "internal: fused step changed kernel");
            continue;
        }
        const bool cuda_core_gemm =
            is_tiled_kind(S.desc.kind) || S.desc.kind == kKindPackF32 || is_direct_kind(S.desc.kind);
        if ((flags & ROSNET_OPT_AUTOTUNE) && cuda_core_gemm &&
            8.0 * (double)S.desc.M * (double)S.desc.N * (double)S.desc.K >= 1e6) {
            // time the candidate kernels on the plan's own operands (contents
            // of intermediates do not matter for timing); C goes to scratch
            auto bptr = [&](int64_t x) -> std::pair<void *, int64_t> {
                if (x < 0) {
                    const Leaf &L = plan->leaves[-1 - x];
                    rosnet_btensor t = nets[L.net].tensors[L.t];
                    return {t->data, t->pstride};
                }
                return {(char *)plan->arena.p + plan->steps[x].arena_off, plan->steps[x].lay.numel};
            };
            DevBuf cs(2 * (size_t)S.lay.numel * (plan->dtype == ROSNET_C64 ? 4 : 8), s);
            GettDesc x = S.desc;
            auto pa = bptr(S.ga), pb = bptr(S.gb);
            bind_operands(x, pa.first, pb.first, cs.p, pa.second, pb.second, S.lay.numel);
            const bool fp32_class = prec != ROSNET_PREC_TF32 && prec != ROSNET_PREC_TF32X3 &&
                                    prec != ROSNET_PREC_BF16X3;
            autotune_problem(x, plan->dtype, fp32_class && (red == kReduceAuto || red == kReduceSequential), red, s);
            S.desc.kind = x.kind;
            S.desc.tiles_m = x.tiles_m;
            S.desc.tiles_n = x.tiles_n;
            S.desc.ksplit = x.ksplit;
            S.desc.ktiles_per_split = x.ktiles_per_split;
            S.desc.flags = (S.desc.flags & ~kFlagStreamK) | (x.flags & kFlagStreamK);   // the tuned schedule
        }
        // tensor-core problems carry their own tensor maps: one launch each
        int key_kind = ((flags & ROSNET_OPT_NOGROUP) || is_packed_kind(S.desc.kind)) ? 1000 + st : S.desc.kind;
        groups[{S.wave, key_kind}].push_back(st);
        // (a packed-operand problem sums its own split in its launch sequence)
        if (S.desc.ksplit > 1 && !(S.desc.flags & kFlagAtomic) && !is_packed_kind(S.desc.kind))
            split_of_wave[S.wave].push_back(st);
        if (S.desc.flags & kFlagAtomic) atomic_of_wave[S.wave].push_back(st);
    }
    // split-K partials: one workspace reused by every wave
    size_t part_bytes = 0;
    for (auto &w : split_of_wave) {
        size_t b = 0;
        for (int st : w.second) b += (desc_part_bytes(plan->steps[st].desc, plan->dtype) + 255) & ~(size_t)255;
        part_bytes = std::max(part_bytes, b);
    }
    if (part_bytes) plan->partials = DevBuf(part_bytes, s);
    for (auto &w : split_of_wave) {
        size_t off = 0;
        for (int st : w.second) {
            plan->steps[st].desc.part = (char *)plan->partials.p + off;
            off += (desc_part_bytes(plan->steps[st].desc, plan->dtype) + 255) & ~(size_t)255;
        }
    }
    std::vector<GettDesc> slot_desc;   // per descriptor slot: the static fields
    size_t tc_bytes = 0;
    auto add_launch = [&](int kind, const std::vector<int> &sts, int role /*0 main 1 reduce 2 zero*/) {
        Plan::Launch L;
        L.kind = kind;
        L.tc_ws_off = 0;
        if (is_packed_kind(kind)) {
            L.tc_ws_off = tc_bytes;
            tc_bytes += (tc_workspace_bytes(plan->steps[sts[0]].desc, packed_mode(kind)) + 255) & ~(size_t)255;
        }
        L.first = (int)plan->desc_step.size();
        L.count = (int)sts.size();
        int64_t ctas = 0;
        for (int st : sts) {
            GettDesc d = plan->steps[st].desc;
            d.tile_begin = ctas;
            ctas += role == 1 ? reduce_ctas(d) : role == 2 ? zero_ctas(d) : desc_ctas(d);
            plan->desc_step.push_back(st);
            slot_desc.push_back(d);
        }
        L.tiles = ctas;
        plan->launches.push_back(L);
    };
    if (!forest_order.empty()) {   // before every wave
        add_launch(kKindForest, forest_order, 0);
        plan->launches.back().tiles = prog[0];
        plan->launches.back().prog_off = prog_off;
    }
    for (auto it = groups.begin(); it != groups.end(); ++it) {
        const int w = it->first.first;
        if ((it == groups.begin() || std::prev(it)->first.first != w) && atomic_of_wave.count(w))
            add_launch(kKindZero, atomic_of_wave[w], 2);   // C = 0 before order-free adds
        add_launch(plan->steps[it->second[0]].desc.kind, it->second, 0);
        auto nx = std::next(it);
        if ((nx == groups.end() || nx->first.first != w) && split_of_wave.count(w))
            add_launch(kKindReduce, split_of_wave[w], 1);
    }
    plan->slot_desc = std::move(slot_desc);
    if (tc_bytes) {   // zeroed once: the stream-K tile counters start at zero
        plan->tcws = DevBuf(tc_bytes, s);
        RN_CHECK_CUDA(cudaMemsetAsync(plan->tcws.p, 0, tc_bytes, s));
    }
    // the launch with the most algorithmic work (8 M N K per complex GEMM)
    {
        const double el2d = 2.0 * (plan->dtype == ROSNET_C64 ? 4 : 8);
        double best = -1;
        for (size_t li = 0; li < plan->launches.size(); ++li) {
            const auto &L = plan->launches[li];
            double fl = 0, by = 0;
            if (L.kind == kKindReduce || L.kind == kKindZero) continue;
            for (int q = L.first; q < L.first + L.count; ++q) {
                const GettDesc &d = plan->slot_desc[q];
                fl += 8.0 * (double)d.M * (double)d.N * (double)d.K;
                by += el2d * ((double)d.M * d.K + (double)d.K * d.N + (double)d.M * d.N);
            }
            if (fl > best) {
                best = fl;
                plan->heavy = (int)li;
                plan->heavy_flops = fl;
                plan->heavy_bytes = by;
                plan->heavy_kind = L.kind;
            }
        }
    }
    const size_t nd = std::max<size_t>(plan->desc_step.size(), 1);
    plan->descs = DevBuf(nd * sizeof(GettDesc), s);
    for (int r = 0; r < Plan::kRing; ++r) {
        RN_CHECK_CUDA(cudaMallocHost((void **)&plan->pinned[r], nd * sizeof(GettDesc)));
        RN_CHECK_CUDA(cudaEventCreateWithFlags(&plan->ev[r], cudaEventDisableTiming));
    }
    RN_CHECK_CUDA(cudaMallocHost((void **)&plan->pinned_small,
                                 (size_t)Plan::kSmallRing * Plan::kSmall * sizeof(GettDesc)));
    for (cudaEvent_t &e : plan->ev_small) RN_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return plan;
}

// Device bytes a plan holds (0 while spilled).
size_t plan_device_bytes(const Plan &P) {
    if (P.spilled) return 0;
    return P.arena.bytes + P.tables.bytes + P.descs.bytes + P.partials.bytes + P.tcws.bytes;
}

// Spill: wait for the plan's work, copy its tables to page-locked host
// memory, release its device buffers and graph.  Returns the host bytes held.
size_t spill_plan(Plan &P, cudaStream_t s) {
    if (P.spilled) return P.tables.bytes;
    RN_CHECK_CUDA(cudaStreamSynchronize(s));
    if (P.side) RN_CHECK_CUDA(cudaStreamSynchronize(P.side));
    for (int i = 0; i < Plan::kRing; ++i)
        if (P.ev[i]) RN_CHECK_CUDA(cudaEventSynchronize(P.ev[i]));
    for (cudaEvent_t e : P.ev_small)
        if (e) RN_CHECK_CUDA(cudaEventSynchronize(e));
    if (P.tables.bytes) {
        if (!P.host_tables) RN_CHECK_CUDA(cudaMallocHost(&P.host_tables, P.tables.bytes));
        RN_CHECK_CUDA(cudaMemcpy(P.host_tables, P.tables.p, P.tables.bytes, cudaMemcpyDeviceToHost));
    }
    P.old_tables = (const char *)P.tables.p;
    P.old_partials = (const char *)P.partials.p;
    if (P.graph) RN_CHECK_CUDA(cudaGraphExecDestroy(P.graph));
    if (P.graph_src) RN_CHECK_CUDA(cudaGraphDestroy(P.graph_src));
    P.graph = nullptr;
    P.graph_src = nullptr;
    for (auto &nd : P.ev_node) nd = nullptr;
    P.arena.reset();
    P.tables.reset();
    P.descs.reset();
    P.partials.reset();
    P.tcws.reset();
    P.mirror_valid = false;
    P.spilled = true;
    return P.tables.bytes;
}

// Restore a spilled plan on stream s: the same buffer sizes again, the tables
// copied back, the descriptors' table and partial-sum pointers moved to the
// new addresses (everything else they hold is bound per call), the graph
// captured again on its next replay.
void restore_plan(Plan &P, cudaStream_t s) {
    if (!P.spilled) return;
    const size_t ab = P.arena.bytes, tb = P.tables.bytes, db = P.descs.bytes, pb = P.partials.bytes,
                 wb = P.tcws.bytes;
    P.arena = DevBuf(ab, s);
    P.tables = DevBuf(tb, s);
    P.descs = DevBuf(db, s);
    P.partials = DevBuf(pb, s);
    P.tcws = DevBuf(wb, s);
    if (tb) RN_CHECK_CUDA(cudaMemcpyAsync(P.tables.p, P.host_tables, tb, cudaMemcpyHostToDevice, s));
    if (wb) RN_CHECK_CUDA(cudaMemsetAsync(P.tcws.p, 0, wb, s));   // stream-K tile counters start at zero
    auto move = [](auto &ptr, const char *from, size_t bytes, void *to) {
        const char *q = (const char *)ptr;
        if (q && from && q >= from && q < from + bytes)
            ptr = (std::remove_reference_t<decltype(ptr)>)((char *)to + (q - from));
    };
    for (GettDesc &d : P.slot_desc) {
        move(d.offAM, P.old_tables, tb, P.tables.p);
        move(d.offCM, P.old_tables, tb, P.tables.p);
        move(d.offBN, P.old_tables, tb, P.tables.p);
        move(d.offCN, P.old_tables, tb, P.tables.p);
        move(d.offAK, P.old_tables, tb, P.tables.p);
        move(d.offBK, P.old_tables, tb, P.tables.p);
        move(d.part, P.old_partials, pb, P.partials.p);
    }
    P.mirror_valid = false;
    P.spilled = false;
}

void run_plan(Plan &P, const rosnet_network *nets, rosnet_btensor *outs, cudaStream_t s) {
    char *arena = (char *)P.arena.p;
    auto leaf_of = [&](int64_t g) -> rosnet_btensor {
        const Leaf &L = P.leaves[-1 - g];
        return nets[L.net].tensors[L.t];
    };
    auto ptr_of = [&](int64_t g) -> void * {
        if (g < 0) return leaf_of(g)->data;
        const Step &S = P.steps[g];
        if (S.arena_off == SIZE_MAX) return outs[S.out_net]->data;
        return arena + S.arena_off;
    };
    auto pstride_of = [&](int64_t g) -> int64_t {
        if (g < 0) return leaf_of(g)->pstride;
        const Step &S = P.steps[g];
        return S.arena_off == SIZE_MAX ? outs[S.out_net]->pstride : S.lay.numel;
    };
    // the stream the plan's work goes on: the caller's, or for a graph
    // requested on the legacy default stream (where graphs cannot be
    // captured) the plan's own stream, ordered after the caller's work
    const bool want_graph = (P.flags & ROSNET_OPT_GRAPH) && !P.launches.empty();
    const cudaStream_t caller = s;
    if (want_graph && s == nullptr) {
        if (!P.side) {
            RN_CHECK_CUDA(cudaStreamCreateWithFlags(&P.side, cudaStreamNonBlocking));
            for (auto &e : P.join) RN_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        }
        RN_CHECK_CUDA(cudaEventRecord(P.join[0], caller));
        RN_CHECK_CUDA(cudaStreamWaitEvent(P.side, P.join[0], 0));
        s = P.side;
    }
    // patch descriptors; stage and upload only the range whose operands
    // changed since the last call.  Only an upload waits (for the copy that
    // last read the pinned staging slot it reuses): a call whose descriptors
    // are unchanged does not hold the host back, and one that changes a few
    // (a new output tensor each call) waits for the upload 64 calls back, so
    // the host can run many calls ahead of the device and a brief host stall
    // leaves the device busy
    const size_t nd = P.desc_step.size();
    if (P.mirror.size() != nd) P.mirror.resize(nd);
    size_t lo = nd, hi = 0;
    for (size_t i = 0; i < nd; ++i) {
        const int st = P.desc_step[i];
        const Step &S = P.steps[st];
        GettDesc d = P.slot_desc[i];
        bind_operands(d, ptr_of(S.ga), ptr_of(S.gb), ptr_of(st), pstride_of(S.ga), pstride_of(S.gb),
                      pstride_of(st));
        const GettDesc &m = P.mirror[i];
        if (!P.mirror_valid || m.a != d.a || m.b != d.b || m.c != d.c || m.a_plane != d.a_plane ||
            m.b_plane != d.b_plane || m.c_plane != d.c_plane) {
            lo = std::min(lo, i);
            hi = i + 1;
            P.mirror[i] = d;
        }
    }
    P.mirror_valid = true;
    if (lo < hi) {
        GettDesc *h;   // the staging slot: the changed range goes to its start
        cudaEvent_t e;
        if (hi - lo <= Plan::kSmall) {
            const int r = P.ring_small;
            P.ring_small = (r + 1) % Plan::kSmallRing;
            h = P.pinned_small + (size_t)r * Plan::kSmall;
            e = P.ev_small[r];
        } else {
            const int r = P.ring;
            P.ring = (r + 1) % Plan::kRing;
            h = P.pinned[r];
            e = P.ev[r];
        }
        RN_CHECK_CUDA(cudaEventSynchronize(e));   // the copy that last read the slot is done
        std::copy(P.mirror.begin() + lo, P.mirror.begin() + hi, h);
        RN_CHECK_CUDA(cudaMemcpyAsync((GettDesc *)P.descs.p + lo, h, (hi - lo) * sizeof(GettDesc),
                                      cudaMemcpyHostToDevice, s));
        RN_CHECK_CUDA(cudaEventRecord(e, s));
    }

    const bool timing = (P.flags & ROSNET_OPT_TIMING) && P.heavy >= 0;
    int slot = -1;
    if (timing) {
        if (P.tev.empty()) {
            P.tev.resize(3 * Plan::kTimingRing, nullptr);
            for (auto &e : P.tev) RN_CHECK_CUDA(cudaEventCreate(&e));
        }
        slot = P.tpos;
        P.tpos = (P.tpos + 1) % Plan::kTimingRing;
    }
    const GettDesc *dd = (const GettDesc *)P.descs.p;
    auto enqueue = [&](bool capturing) {
        for (size_t li = 0; li < P.launches.size(); ++li) {
            const auto &L = P.launches[li];
            const bool th = timing && (int)li == P.heavy;
            // timed: the whole launch (operand packs included) and, for a
            // packed-operand launch, its GEMM kernel alone
            auto rec = [&](int which) {
                cudaEvent_t e = P.tev[3 * slot + which];
                RN_CHECK_CUDA(capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                        : cudaEventRecord(e, s));
            };
            if (th) rec(0);
            if (is_packed_kind(L.kind)) {
                GroupArgs ga;
                memset(&ga, 0, sizeof(ga));
                ga.descs = dd + L.first;
                ga.ndesc = 1;
                std::function<void()> hook;
                if (th) hook = [&]() { rec(1); };
                // the host copy carries the operand addresses that tensor maps
                // over operands read in place are encoded with (only arena
                // intermediates are flagged dense: their addresses are fixed
                // for the life of the plan, so a captured graph stays valid)
                const int st = P.desc_step[L.first];
                const Step &S = P.steps[st];
                GettDesc x = P.slot_desc[L.first];
                bind_operands(x, ptr_of(S.ga), ptr_of(S.gb), ptr_of(st), pstride_of(S.ga), pstride_of(S.gb),
                              pstride_of(st));
                launch_tc_problem(packed_mode(L.kind), x, ga, (char *)P.tcws.p + L.tc_ws_off, s, true, true, hook);
            } else if (L.kind == kKindForest) {
                launch_forest(P.dtype, dd + L.first, (const int64_t *)P.tables.p + L.prog_off, L.tiles, s);
            } else {
                launch_gett_group(L.kind, P.dtype, dd + L.first, L.count, L.tiles, s);
            }
            if (th) rec(2);
        }
    };
    const bool use_graph = want_graph && s != nullptr;
    if (use_graph) {
        if (!P.graph) {
            cudaGraph_t gr = nullptr;
            RN_CHECK_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            int64_t before = g_launches.load();
            try {
                enqueue(true);
            } catch (...) {
                cudaStreamEndCapture(s, &gr);
                if (gr) cudaGraphDestroy(gr);
                throw;
            }
            P.graph_nodes = (int)(g_launches.load() - before);
            g_launches -= P.graph_nodes;  // counted at replay
            RN_CHECK_CUDA(cudaStreamEndCapture(s, &gr));
            if (timing) {  // find the event-record nodes (two, or three for a packed launch)
                size_t nn = 0;
                RN_CHECK_CUDA(cudaGraphGetNodes(gr, nullptr, &nn));
                std::vector<cudaGraphNode_t> nodes(nn);
                RN_CHECK_CUDA(cudaGraphGetNodes(gr, nodes.data(), &nn));
                for (auto nd_ : nodes) {
                    cudaGraphNodeType ty;
                    RN_CHECK_CUDA(cudaGraphNodeGetType(nd_, &ty));
                    if (ty != cudaGraphNodeTypeEventRecord) continue;
                    cudaEvent_t e;
                    RN_CHECK_CUDA(cudaGraphEventRecordNodeGetEvent(nd_, &e));
                    for (int w = 0; w < 3; ++w)
                        if (e == P.tev[3 * slot + w]) P.ev_node[w] = nd_;
                }
            }
            cudaError_t e = cudaGraphInstantiate(&P.graph, gr, 0);
            P.graph_src = gr;
            RN_CHECK_CUDA(e);
        } else if (timing) {
            for (int w = 0; w < 3; ++w)
                if (P.ev_node[w])
                    RN_CHECK_CUDA(cudaGraphExecEventRecordNodeSetEvent(P.graph, P.ev_node[w], P.tev[3 * slot + w]));
        }
        RN_CHECK_CUDA(cudaGraphLaunch(P.graph, s));
        g_launches += P.graph_nodes;
    } else {
        enqueue(false);
    }
    if (timing) {
        g_timing_log.push_back({&P, slot});
        // a drain reports only the newest kTimingRing entries: keep the log
        // bounded for callers that time without draining
        if (g_timing_log.size() > 2 * (size_t)Plan::kTimingRing)
            g_timing_log.erase(g_timing_log.begin(), g_timing_log.end() - Plan::kTimingRing);
    }
    // results that are not written in place: permuted, shared, or a lone leaf
    for (int i = 0; i < P.nnet; ++i) {
        const NetOut &O = P.outs[i];
        if (O.direct) continue;
        const Layout &src = O.final_gid >= 0 ? P.steps[O.final_gid].lay : leaf_of(O.final_gid)->lay;
        launch_relayout(src, outs[i]->lay, O.perm.data(), P.dtype, ptr_of(O.final_gid),
                        pstride_of(O.final_gid), outs[i]->data, outs[i]->pstride, s);
    }
    if (s != caller) {   // the caller's later work sees the results
        RN_CHECK_CUDA(cudaEventRecord(P.join[1], s));
        RN_CHECK_CUDA(cudaStreamWaitEvent(caller, P.join[1], 0));
    }
}

}  // namespace

}  // namespace rosnet

using namespace rosnet;

extern "C" {

static void precheck_network(const rosnet_network *net, const rosnet_path *path) {
    if (!net || net->ntensors < 1 || !net->tensors || !net->ranks || !net->labels)
        RN_FAIL(ROSNET_ERR_INVALID_ARG, "malformed network");
    for (int t = 0; t < net->ntensors; ++t)
        if (!net->tensors[t] || net->ranks[t] != net->tensors[t]->lay.rank ||
            (net->ranks[t] > 0 && !net->labels[t]))
            RN_FAIL(ROSNET_ERR_INVALID_ARG, "NULL tensor or rank mismatch in network");
    if (net->nout < 0 || (net->nout > 0 && !net->out_labels))
        RN_FAIL(ROSNET_ERR_INVALID_ARG, "malformed output labels");
    if (!path || path->nsteps < 0 || (path->nsteps > 0 && !path->pairs))
        RN_FAIL(ROSNET_ERR_INVALID_ARG, "NULL path");
}

static void contract_batch(int nnet, const rosnet_network *nets, const rosnet_path *paths,
                           const rosnet_opts *opts, cudaStream_t s, rosnet_btensor *outs) {
    if (nnet < 1 || !nets || !paths) RN_FAIL(ROSNET_ERR_INVALID_ARG, "no networks");
    for (int i = 0; i < nnet; ++i) precheck_network(&nets[i], &paths[i]);
    const int prec = check_precision(opts, nets[0].tensors[0]->dtype);
    const int flags = opts ? opts->flags : 0;
    (void)check_reduce(opts);
    const int64_t maxblk = opts ? opts->max_block_entries : 0;
    if (maxblk < 0) RN_FAIL(ROSNET_ERR_INVALID_ARG, "negative max_block_entries");
    std::vector<Leaf> leaves;
    auto slot = leaf_slots(nnet, nets, &leaves);
    Key128 key = plan_key(nnet, nets, paths, slot, prec, flags, maxblk, s);
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plans.find(key);
    Plan *P;
    if (it == g_plans.end()) {
        for (int i = 0; i < nnet; ++i) validate_network(&nets[i]);  // the key encodes all of it
        auto np = build_plan(nnet, nets, paths, slot, std::move(leaves), prec, flags, maxblk, s);
        if (g_plan_limit > 0) evict_plans_to((size_t)g_plan_limit - 1);
        P = np.get();
        g_plans.emplace(std::move(key), std::move(np));
    } else {
        P = it->second.get();
        P->leaves = std::move(leaves);   // same sharing pattern; refresh the representatives
        restore_plan(*P, s);
    }
    P->last_used = ++g_plan_clock;
    std::vector<rosnet_btensor> made;
    try {
        for (int i = 0; i < nnet; ++i) {
            const Layout &L = P->outs[i].out_lay;
            made.push_back(new_tensor(L.rank, L.shape, L.block, P->dtype, s));
        }
        run_plan(*P, nets, made.data(), s);
    } catch (...) {
        for (auto t : made) free_tensor(t);
        throw;
    }
    for (int i = 0; i < nnet; ++i) outs[i] = made[i];
}

rosnet_status rosnet_contract(const rosnet_network *net, const rosnet_path *path,
                              const rosnet_opts *opts, void *stream, rosnet_btensor *out) {
    if (!out) return ROSNET_ERR_INVALID_ARG;
    *out = nullptr;
    RN_API_BEGIN
    contract_batch(1, net, path, opts, (cudaStream_t)stream, out);
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_contract_batch(int32_t nnet, const rosnet_network *nets, const rosnet_path *paths,
                                    const rosnet_opts *opts, void *stream, rosnet_btensor *outs) {
    if (!outs || nnet < 1) return ROSNET_ERR_INVALID_ARG;
    for (int i = 0; i < nnet; ++i) outs[i] = nullptr;
    RN_API_BEGIN
    contract_batch(nnet, nets, paths, opts, (cudaStream_t)stream, outs);
    return ROSNET_OK;
    RN_API_END
}

// The cache key of the plan rosnet_contract_batch would use for these arguments.
static Key128 cached_key(int32_t nnet, const rosnet_network *nets, const rosnet_path *paths,
                         const rosnet_opts *opts, void *stream) {
    if (nnet < 1 || !nets || !paths) RN_FAIL(ROSNET_ERR_INVALID_ARG, "no networks");
    for (int i = 0; i < nnet; ++i) precheck_network(&nets[i], &paths[i]);
    const int prec = check_precision(opts, nets[0].tensors[0]->dtype);
    const int flags = opts ? opts->flags : 0;
    const int64_t maxblk = opts ? opts->max_block_entries : 0;
    std::vector<Leaf> leaves;
    auto slot = leaf_slots(nnet, nets, &leaves);
    return plan_key(nnet, nets, paths, slot, prec, flags, maxblk, (cudaStream_t)stream);
}

rosnet_status rosnet_plan_stats(int32_t nnet, const rosnet_network *nets, const rosnet_path *paths,
                                const rosnet_opts *opts, void *stream, int64_t *steps_requested,
                                int64_t *steps_planned, int64_t *launches, int64_t *packed_operands,
                                int64_t *device_bytes) {
    RN_API_BEGIN
    Key128 key = cached_key(nnet, nets, paths, opts, stream);
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plans.find(key);
    if (it == g_plans.end()) RN_FAIL(ROSNET_ERR_INVALID_ARG, "no cached plan for these networks");
    if (device_bytes) *device_bytes = (int64_t)plan_device_bytes(*it->second);
    if (steps_requested) *steps_requested = it->second->steps_requested;
    if (steps_planned) *steps_planned = (int64_t)it->second->steps.size();
    if (launches) *launches = (int64_t)it->second->launches.size();
    if (packed_operands) {
        int64_t n = 0;
        const Plan &P = *it->second;
        for (const auto &L : P.launches) {
            if (!is_packed_kind(L.kind)) continue;
            const int f = P.slot_desc[L.first].flags;
            const bool f32 = L.kind == kKindPackF32;
            n += (f32 && (f & kFlagADense)) ? 0 : 1;
            n += (f32 && (f & kFlagBDense)) ? 0 : 1;
        }
        *packed_operands = n;
    }
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_timing_drain(double *ms, double *ms_whole, double *flops, double *bytes,
                                  int32_t *kinds, int32_t max_entries, int32_t *n) {
    if (!n || max_entries < 0 || (max_entries > 0 && !ms)) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    std::lock_guard<std::mutex> lk(g_plan_mu);
    int32_t k = 0;
    // keep only the newest kTimingRing entries per plan (older slots were reused)
    size_t start = g_timing_log.size() > (size_t)Plan::kTimingRing
                       ? g_timing_log.size() - Plan::kTimingRing : 0;
    for (size_t i = start; i < g_timing_log.size() && k < max_entries; ++i) {
        Plan *P = g_timing_log[i].first;
        int slot = g_timing_log[i].second;
        RN_CHECK_CUDA(cudaEventSynchronize(P->tev[3 * slot + 2]));
        const bool packed = is_packed_kind(P->heavy_kind);
        float t = 0, tw = 0;
        RN_CHECK_CUDA(cudaEventElapsedTime(&t, P->tev[3 * slot + (packed ? 1 : 0)], P->tev[3 * slot + 2]));
        RN_CHECK_CUDA(cudaEventElapsedTime(&tw, P->tev[3 * slot], P->tev[3 * slot + 2]));
        ms[k] = t;
        if (ms_whole) ms_whole[k] = tw;
        if (flops) flops[k] = P->heavy_flops;
        if (bytes) bytes[k] = P->heavy_bytes;
        if (kinds) kinds[k] = P->heavy_kind;
        ++k;
    }
    g_timing_log.clear();
    *n = k;
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_plan_cache_limit(int32_t max_plans, int32_t *cached) {
    RN_API_BEGIN
    std::lock_guard<std::mutex> lk(g_plan_mu);
    if (max_plans >= 0) {
        g_plan_limit = max_plans;
        if (max_plans > 0) evict_plans_to((size_t)max_plans);
    }
    if (cached) *cached = (int32_t)g_plans.size();
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_plan_release(int32_t nnet, const rosnet_network *nets, const rosnet_path *paths,
                                  const rosnet_opts *opts, void *stream) {
    RN_API_BEGIN
    Key128 key = cached_key(nnet, nets, paths, opts, stream);
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plans.find(key);
    if (it == g_plans.end()) RN_FAIL(ROSNET_ERR_INVALID_ARG, "no cached plan for these networks");
    Plan *vp = it->second.get();
    g_timing_log.erase(std::remove_if(g_timing_log.begin(), g_timing_log.end(),
                                      [vp](const std::pair<Plan *, int> &e) { return e.first == vp; }),
                       g_timing_log.end());
    g_plans.erase(it);
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_plan_spill(int32_t nnet, const rosnet_network *nets, const rosnet_path *paths,
                                const rosnet_opts *opts, void *stream, int64_t *host_bytes) {
    RN_API_BEGIN
    Key128 key = cached_key(nnet, nets, paths, opts, stream);
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plans.find(key);
    if (it == g_plans.end()) RN_FAIL(ROSNET_ERR_INVALID_ARG, "no cached plan for these networks");
    const size_t hb = spill_plan(*it->second, (cudaStream_t)stream);
    if (host_bytes) *host_bytes = (int64_t)hb;
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_release_plans(void) {
    RN_API_BEGIN
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_timing_log.clear();
    g_plans.clear();
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_path_greedy_extents(int32_t ntensors, const int32_t *ranks,
                                         const int64_t *const *labels, const int64_t *const *extents,
                                         int32_t nout, const int64_t *out_labels, int32_t *pairs_out,
                                         int32_t *nsteps) {
    if (!pairs_out || !nsteps || ntensors < 1 || !ranks || !labels || !extents ||
        (nout > 0 && !out_labels) || nout < 0)
        return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    const int nt = ntensors;
    std::unordered_map<int64_t, int64_t> ext;  // label -> extent
    std::vector<std::vector<int64_t>> lab(2 * nt);
    std::vector<bool> alive(2 * nt, false);
    std::unordered_map<int64_t, std::vector<int>> holders;  // label -> live ids carrying it
    for (int t = 0; t < nt; ++t) {
        if (ranks[t] < 0 || ranks[t] > kMaxRank) RN_FAIL(ROSNET_ERR_RANK_LIMIT, "bad rank");
        if (ranks[t] > 0 && (!labels[t] || !extents[t])) RN_FAIL(ROSNET_ERR_INVALID_ARG, "NULL labels");
        lab[t].assign(labels[t], labels[t] + ranks[t]);
        alive[t] = true;
        for (int i = 0; i < ranks[t]; ++i) {
            int64_t e = extents[t][i];
            auto it = ext.find(lab[t][i]);
            if (it != ext.end() && it->second != e)
                RN_FAIL(ROSNET_ERR_SHAPE, "a label has two different extents");
            ext[lab[t][i]] = e;
            holders[lab[t][i]].push_back(t);
        }
    }
    for (auto &kv : holders)
        if (kv.second.size() > 2) RN_FAIL(ROSNET_ERR_UNSUPPORTED, "a label carried by more than two tensors");
    auto size_of = [&](const std::vector<int64_t> &l) {
        double s = 1;
        for (int64_t x : l) s *= (double)ext[x];
        return s;
    };
    auto result_labels = [&](int a, int b) {
        std::vector<int64_t> r;
        for (int64_t x : lab[a])
            if (std::find(lab[b].begin(), lab[b].end(), x) == lab[b].end()) r.push_back(x);
        for (int64_t x : lab[b])
            if (std::find(lab[a].begin(), lab[a].end(), x) == lab[a].end()) r.push_back(x);
        return r;
    };
    int next = nt;
    for (int st = 0; st < nt - 1; ++st) {
        bool found = false;
        double best_size = 0, best_delta = 0;
        int ba = -1, bb = -1;
        for (auto &kv : holders) {
            const auto &h = kv.second;
            if (h.size() != 2) continue;
            int a = std::min(h[0], h[1]), b = std::max(h[0], h[1]);
            std::vector<int64_t> r = result_labels(a, b);
            double sz = size_of(r);
            double delta = sz - size_of(lab[a]) - size_of(lab[b]);
            bool better = !found || sz < best_size ||
                          (sz == best_size && (delta < best_delta ||
                                               (delta == best_delta && (a < ba || (a == ba && b < bb)))));
            if (better) {
                found = true;
                best_size = sz;
                best_delta = delta;
                ba = a;
                bb = b;
            }
        }
        if (!found) {  // disconnected: outer product of the two lowest live ids
            for (int i = 0; i < next && bb < 0; ++i)
                if (alive[i]) { if (ba < 0) ba = i; else bb = i; }
        }
        std::vector<int64_t> r = result_labels(ba, bb);
        for (int64_t x : lab[ba]) {
            auto &h = holders[x];
            h.erase(std::remove(h.begin(), h.end(), ba), h.end());
        }
        for (int64_t x : lab[bb]) {
            auto &h = holders[x];
            h.erase(std::remove(h.begin(), h.end(), bb), h.end());
        }
        alive[ba] = alive[bb] = false;
        lab[next] = r;
        alive[next] = true;
        for (int64_t x : r) holders[x].push_back(next);
        pairs_out[2 * st] = ba;
        pairs_out[2 * st + 1] = bb;
        ++next;
    }
    *nsteps = nt - 1;
    return ROSNET_OK;
    RN_API_END
}

// ---------------------------------------------------------------------------
// host-side path and slicing heuristics
// ---------------------------------------------------------------------------
namespace {

// A network's labels renumbered 0..L-1 (in order of first appearance) with
// their extents.  Membership of a label in a tensor is tested with a stamp
// array instead of a scan; every product below is still taken over the same
// labels in the same order, so costs are the same doubles as a plain scan
// would give.
struct LabelNet {
    int nt;
    std::vector<std::vector<int64_t>> lab;   // original labels per tensor
    std::vector<std::vector<int>> id;        // the same as dense ids
    std::vector<int64_t> label;              // dense id -> label
    std::vector<double> ext;                 // dense id -> extent
    std::unordered_map<int64_t, int> dense;  // label -> dense id
};

LabelNet label_net(int32_t ntensors, const int32_t *ranks, const int64_t *const *labels,
                   const int64_t *const *extents) {
    if (ntensors < 1 || !ranks || !labels || !extents) RN_FAIL(ROSNET_ERR_INVALID_ARG, "malformed network");
    LabelNet n;
    n.nt = ntensors;
    n.lab.resize(ntensors);
    n.id.resize(ntensors);
    std::vector<int> cnt;
    for (int t = 0; t < ntensors; ++t) {
        if (ranks[t] < 0 || ranks[t] > kMaxRank) RN_FAIL(ROSNET_ERR_RANK_LIMIT, "bad rank");
        if (ranks[t] > 0 && (!labels[t] || !extents[t])) RN_FAIL(ROSNET_ERR_INVALID_ARG, "NULL labels");
        n.lab[t].assign(labels[t], labels[t] + ranks[t]);
        for (int i = 0; i < ranks[t]; ++i) {
            auto ins = n.dense.emplace(labels[t][i], (int)n.label.size());
            if (ins.second) {
                n.label.push_back(labels[t][i]);
                n.ext.push_back((double)extents[t][i]);
                cnt.push_back(0);
            }
            const int x = ins.first->second;
            if (n.ext[x] != (double)extents[t][i]) RN_FAIL(ROSNET_ERR_SHAPE, "a label has two different extents");
            if (++cnt[x] > 2) RN_FAIL(ROSNET_ERR_UNSUPPORTED, "a label carried by more than two tensors");
            n.id[t].push_back(x);
        }
    }
    return n;
}

// Stamps for membership tests: mark(l) tags the labels of l, and has(x) is
// true for those labels until the next mark().
struct Marks {
    std::vector<uint32_t> m;
    uint32_t tok = 0;
    explicit Marks(size_t n) : m(n, 0) {}
    void mark(const std::vector<int> &l) {
        if (++tok == 0) {   // wrapped: clear the stamps once
            std::fill(m.begin(), m.end(), 0);
            tok = 1;
        }
        for (int x : l) m[x] = tok;
    }
    bool has(int x) const { return m[x] == tok; }
};

// Entries of a tensor: the product of its extents in label order.
double entries(const LabelNet &n, const std::vector<int> &l) {
    double v = 1;
    for (int x : l) v *= n.ext[x];
    return v;
}

// Labels of the result of joining a and b: a's labels not in b, then b's
// not in a.
void joined(const std::vector<int> &a, const std::vector<int> &b, Marks &mk, std::vector<int> &r) {
    r.clear();
    mk.mark(b);
    for (int x : a)
        if (!mk.has(x)) r.push_back(x);
    mk.mark(a);
    for (int x : b)
        if (!mk.has(x)) r.push_back(x);
}

// A path in SSA form (step t joins two live ids and creates id nt + t): every
// id in range, the two ids of a step distinct, and each id used once.
void check_ssa_path(int nt, const int32_t *pairs, int nsteps) {
    if (nsteps != nt - 1 || (nsteps > 0 && !pairs)) RN_FAIL(ROSNET_ERR_INVALID_ARG, "a path must have ntensors - 1 steps");
    std::vector<char> used(nt + nsteps, 0);
    for (int st = 0; st < nsteps; ++st) {
        const int32_t a = pairs[2 * st], b = pairs[2 * st + 1];
        if (a < 0 || b < 0 || a >= nt + st || b >= nt + st || a == b || used[a] || used[b])
            RN_FAIL(ROSNET_ERR_INVALID_ARG, "path step " + std::to_string(st) + " uses a dead or unknown id");
        used[a] = used[b] = 1;
    }
}

// Max intermediate entries and total 8*M*N*K flops of a path, with the
// labels flagged in `cut` (by dense id) fixed (sliced: extent 1).  `live`
// is scratch reused between calls.
std::pair<double, double> path_cost(const LabelNet &n, const int32_t *pairs, int nsteps,
                                    const std::vector<char> &cut, Marks &mk,
                                    std::vector<std::vector<int>> &live) {
    auto e = [&](int x) { return cut.empty() || !cut[x] ? n.ext[x] : 1.0; };
    if (live.size() < (size_t)(n.nt + nsteps)) live.resize(n.nt + nsteps);
    for (int t = 0; t < n.nt; ++t) live[t] = n.id[t];
    double mx = 0, tot = 0;
    for (int st = 0; st < nsteps; ++st) {
        const auto &la = live[pairs[2 * st]], &lb = live[pairs[2 * st + 1]];
        auto &lc = live[n.nt + st];
        lc.clear();
        double all = 1, out = 1;
        mk.mark(lb);
        for (int x : la) {
            all *= e(x);
            if (!mk.has(x)) { lc.push_back(x); out *= e(x); }
        }
        mk.mark(la);
        for (int x : lb)
            if (!mk.has(x)) { lc.push_back(x); out *= e(x); all *= e(x); }
        tot += 8.0 * all;
        mx = std::max(mx, out);
    }
    return {mx, tot};
}

// The bonds of a network in the order in which a label -> holders hash map,
// filled tensor by tensor and label by label, visits its keys (dense ids).
// Trials of the randomised search visit candidates in this order.
std::vector<int> visit_order(const LabelNet &n) {
    std::unordered_map<int64_t, std::vector<int>> holders;
    for (int t = 0; t < n.nt; ++t)
        for (int64_t x : n.lab[t]) holders[x].push_back(t);
    std::vector<int> order;
    order.reserve(holders.size());
    for (const auto &kv : holders) order.push_back(n.dense.at(kv.first));
    return order;
}

}  // namespace

rosnet_status rosnet_path_search(int32_t ntensors, const int32_t *ranks, const int64_t *const *labels,
                                 const int64_t *const *extents, int32_t nout, const int64_t *out_labels,
                                 int32_t ntrials, uint64_t seed, double temperature, int32_t *pairs_out,
                                 int32_t *nsteps, double *flops) {
    if (!pairs_out || !nsteps || ntrials < 1 || temperature < 0) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    LabelNet n = label_net(ntensors, ranks, labels, extents);
    Marks mk(n.ext.size());
    const int ns = ntensors - 1;
    // trial 0: the deterministic greedy min-size path
    std::vector<int32_t> best(2 * std::max(ns, 0)), cur(2 * std::max(ns, 0));
    int32_t k = 0;
    rosnet_status rc = rosnet_path_greedy_extents(ntensors, ranks, labels, extents, nout, out_labels,
                                                  best.data(), &k);
    if (rc != ROSNET_OK) return rc;
    std::vector<std::vector<int>> scratch0;
    double best_flops = path_cost(n, best.data(), ns, {}, mk, scratch0).second;
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U(1e-12, 1.0);
    std::vector<int> r;
    std::vector<std::vector<int>> scratch;
    const std::vector<int> order = visit_order(n);
    // holders of each label (at most two live tensors carry it), in the order
    // they took it up
    struct Hold {
        int t[2];
        int k;
        void drop(int v) {   // remove every occurrence of v, keeping the rest in order
            int w = 0;
            for (int i = 0; i < k; ++i)
                if (t[i] != v) t[w++] = t[i];
            k = w;
        }
        void add(int v) {
            if (k >= 2) RN_FAIL(ROSNET_ERR_UNSUPPORTED, "a label carried by more than two tensors");
            t[k++] = v;
        }
    };
    for (int trial = 1; trial < ntrials; ++trial) {
        // greedy on cost = size(out) - size(a) - size(b), perturbed by Gumbel
        // noise of relative scale `temperature`, candidates in visit order
        std::vector<std::vector<int>> live(2 * ntensors);
        std::vector<double> size(2 * ntensors, 1.0);
        std::vector<Hold> hold(n.ext.size(), Hold{{-1, -1}, 0});
        // size(out) - size(a) - size(b) of each bond's pair, kept until one
        // of the pair is joined (it depends on the two tensors alone)
        std::vector<double> base(n.ext.size(), 0.0);
        std::vector<char> fresh(n.ext.size(), 0);
        std::vector<bool> alive(2 * ntensors, false);
        for (int t = 0; t < ntensors; ++t) {
            live[t] = n.id[t];
            size[t] = entries(n, live[t]);
            alive[t] = true;
            for (int x : live[t]) hold[x].add(t);
        }
        int next = ntensors;
        for (int st = 0; st < ns; ++st) {
            double bc = 0;
            int ba = -1, bb = -1;
            for (int lx : order) {
                const Hold &h = hold[lx];
                if (h.k != 2) continue;
                const int a = std::min(h.t[0], h.t[1]), b = std::max(h.t[0], h.t[1]);
                if (!fresh[lx]) {
                    double out = 1;
                    mk.mark(live[b]);
                    for (int x : live[a])
                        if (!mk.has(x)) out *= n.ext[x];
                    mk.mark(live[a]);
                    for (int x : live[b])
                        if (!mk.has(x)) out *= n.ext[x];
                    base[lx] = out - size[a] - size[b];
                    fresh[lx] = 1;
                }
                double c = base[lx];
                c -= temperature * std::log(-std::log(U(rng))) * std::max(1.0, std::fabs(c));
                if (ba < 0 || c < bc || (c == bc && (a < ba || (a == ba && b < bb)))) { bc = c; ba = a; bb = b; }
            }
            if (ba < 0)   // disconnected: the two lowest live ids
                for (int i = 0; i < next && bb < 0; ++i)
                    if (alive[i]) { if (ba < 0) ba = i; else bb = i; }
            joined(live[ba], live[bb], mk, r);
            for (int x : live[ba]) hold[x].drop(ba);
            for (int x : live[bb]) hold[x].drop(bb);
            alive[ba] = alive[bb] = false;
            live[next] = r;
            size[next] = entries(n, r);
            alive[next] = true;
            for (int x : r) {
                hold[x].add(next);
                fresh[x] = 0;   // its pair now includes the new tensor
            }
            cur[2 * st] = ba;
            cur[2 * st + 1] = bb;
            ++next;
        }
        const double f = path_cost(n, cur.data(), ns, {}, mk, scratch).second;
        if (f < best_flops) { best_flops = f; best = cur; }
    }
    std::copy(best.begin(), best.end(), pairs_out);
    *nsteps = ns;
    if (flops) *flops = best_flops;
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_slice_search(int32_t ntensors, const int32_t *ranks, const int64_t *const *labels,
                                  const int64_t *const *extents, int32_t nout, const int64_t *out_labels,
                                  int32_t nsteps, const int32_t *pairs, int32_t nslice, int64_t *chosen,
                                  double *max_entries, double *flops) {
    if (!chosen || nslice < 0 || !pairs || nsteps != ntensors - 1 || (nout > 0 && !out_labels))
        return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    LabelNet n = label_net(ntensors, ranks, labels, extents);
    check_ssa_path(ntensors, pairs, nsteps);
    Marks mk(n.ext.size());
    std::vector<std::vector<int>> scratch;
    std::unordered_map<int64_t, int> cnt;
    for (auto &l : n.lab) for (int64_t x : l) cnt[x]++;
    std::vector<int64_t> bonds;
    for (auto &kv : cnt) {
        bool is_out = false;
        for (int o = 0; o < nout; ++o) is_out |= out_labels[o] == kv.first;
        if (kv.second == 2 && !is_out) bonds.push_back(kv.first);
    }
    std::sort(bonds.begin(), bonds.end());
    if ((size_t)nslice > bonds.size()) RN_FAIL(ROSNET_ERR_INVALID_ARG, "more slices than bonds");
    std::vector<char> cut(n.ext.size(), 0);   // by dense id
    std::vector<int64_t> order;               // the chosen labels, in order
    std::pair<double, double> cost = path_cost(n, pairs, nsteps, cut, mk, scratch);
    for (int r = 0; r < nslice; ++r) {
        int64_t bl = 0;
        std::pair<double, double> bc{0, 0};
        bool have = false;
        for (int64_t b : bonds) {
            const int x = n.dense.at(b);
            if (cut[x]) continue;
            cut[x] = 1;
            auto c = path_cost(n, pairs, nsteps, cut, mk, scratch);
            cut[x] = 0;
            // the slice count multiplies the flops by the sliced extent
            c.second *= n.ext[x];
            if (!have || c < bc) { bc = c; bl = b; have = true; }
        }
        cut[n.dense.at(bl)] = 1;
        order.push_back(bl);
        cost = bc;
        chosen[r] = bl;
    }
    if (max_entries) *max_entries = path_cost(n, pairs, nsteps, cut, mk, scratch).first;
    if (flops) {
        double mult = 1;
        for (int64_t x : order) mult *= n.ext[n.dense.at(x)];
        *flops = path_cost(n, pairs, nsteps, cut, mk, scratch).second * mult;
    }
    return ROSNET_OK;
    RN_API_END
}

rosnet_status rosnet_path_greedy(const rosnet_network *net, int32_t *pairs_out, int32_t *nsteps) {
    if (!pairs_out || !nsteps) return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    validate_network(net);
    std::vector<const int64_t *> ex(net->ntensors);
    for (int t = 0; t < net->ntensors; ++t) ex[t] = net->tensors[t]->lay.shape;
    return rosnet_path_greedy_extents(net->ntensors, net->ranks, net->labels, ex.data(), net->nout,
                                      net->out_labels, pairs_out, nsteps);
    RN_API_END
}

}  // extern "C"
