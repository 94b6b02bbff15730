// C ABI of libvelopir.so (declared in include/velopir.h): context, key upload,
// layer-batched execution of gate programs, the three VeLoPIR query modes and
// the continuous-batching serving loop.
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/velopir.h"
#include "sched.h"
#include "vp_internal.h"

using namespace vp;

static_assert(sizeof(velopir_trace_rec) == (size_t)kTraceWords * 4, "trace record layout");
static_assert(VELOPIR_TRACE_MAX_IN == kSumMax, "trace record inputs");

namespace {

thread_local std::string g_create_error;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct ServeQuery;

}  // namespace

struct velopir_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;      // 0 = unlimited
    size_t allocated = 0;   // bytes currently held
    std::mutex err_mu;      // guards err: the issue thread and the caller may both fail
    std::string err;
    uint64_t launches = 0;
    int path = VP_PATH_NTT;
    int big_rows = 1 << 16; // blind rotations per launch at most (extracted-row scratch)
    int enc_fanin = 2;      // fan-in of the *_encdb calls' XOR aggregation tree

    bool key_loaded = false;
    DevBuf bk, ksk, bk_ntt, big, jobs_br, jobs_ks, jobs_fr, jobs_sm, jobs_tr, pool, in, out, errw;
    bool bk_ntt_ready = false;
    DevBuf bk_tc, tc_scratch;               // tensor-core path: expanded key, per-launch scratch
    bool bk_tc_ready = false;

    // gate trace (velopir_trace_start / _stop): of a chunk of G gates,
    // max(min(per_launch, G), ceil(G / one_in)) chosen by a seeded generator
    // are copied into trace_buf
    bool trace_on = false;
    uint64_t trace_rng = 0;
    uint32_t trace_per_launch = 0, trace_one_in = 0;
    size_t trace_cap = 0, trace_next = 0;
    DevBuf trace_buf;

    std::deque<std::unique_ptr<ServeQuery>> waiting;
    std::vector<std::unique_ptr<ServeQuery>> active;
    std::vector<std::unique_ptr<ServeQuery>> finished;
    uint64_t next_ticket = 1;
    size_t serve_reserved = 0;

    // issue thread (velopir_serve_start): guards the serving state above
    std::mutex mu;
    std::thread issuer;
    std::atomic<bool> serving{false};
    bool stop_req = false;
    int issuer_rc = VELOPIR_OK;           // first failure of the issue thread
    std::string issuer_err;
    struct Step { cudaEvent_t ev; int *err; };
    std::deque<Step> inflight;            // issued serving steps, oldest first
    int *err_host = nullptr;              // pinned copies of the error word, one per in-flight step
    DevBuf s_br, s_ks, s_fr, s_sm, s_tr;   // serving-step job buffers

    // tracing: events around each launch, resolved lazily
    bool prof = false;
    struct Rec { int kind; uint64_t units; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> spare;
    uint64_t prof_launches[5] = {0, 0, 0, 0, 0}, prof_units[5] = {0, 0, 0, 0, 0};
    double prof_ms[5] = {0, 0, 0, 0, 0};

    // captured launch sequence of the last graph-mode program, replayed when
    // the next one has the same launch list on the same buffers
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<uint64_t> graph_sig;
    uint64_t graph_replays = 0;
};

namespace {

int fail(velopir_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        std::lock_guard<std::mutex> g(c->err_mu);
        c->err = buf;
    } else {
        g_create_error = buf;
    }
    return code;
}

std::string last_error_of(velopir_ctx *c)
{
    std::lock_guard<std::mutex> g(c->err_mu);
    return c->err;
}

#define CU(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(c, VELOPIR_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

void dev_free(velopir_ctx *c, DevBuf &b)
{
    if (b.p) {
        cudaFree(b.p);
        c->allocated -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

// Grow-only device buffer, accounted against the HBM budget.
int ensure(velopir_ctx *c, DevBuf &b, size_t bytes)
{
    if (bytes <= b.bytes) return VELOPIR_OK;
    bytes = std::max(bytes, b.bytes + b.bytes / 2);
    if (c->budget && c->allocated - b.bytes + bytes > c->budget)
        return fail(c, VELOPIR_ERR_OOM, "HBM budget of %zu bytes exceeded (need %zu more)", c->budget,
                    bytes - b.bytes);
    if (b.p) {
        cudaStreamSynchronize(c->stream);
        dev_free(c, b);
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, VELOPIR_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    b.p = p;
    b.bytes = bytes;
    c->allocated += bytes;
    return VELOPIR_OK;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T> T *as(const DevBuf &b) { return reinterpret_cast<T *>(b.p); }

uint32_t *resolve(uint64_t v, uint32_t *pool, const std::vector<int> &phys)
{
    if (!(v & kSlotTag)) return reinterpret_cast<uint32_t *>(v);
    return pool + (size_t)phys[(size_t)(v & ~kSlotTag)] * kSlotWords;
}

struct Launch {
    int kind;   // 0 = blind rotation, 1 = key switch, 2 = free gates, 3 = pre-combination sums, 4 = gate trace
    size_t off;
    int n;
};

struct Flat {
    std::vector<BrJob> br;
    std::vector<KsJob> ks;
    std::vector<FreeJob> fr;
    std::vector<SumJob> sm;
    std::vector<TraceJob> tr;
    std::vector<Launch> launches;
};

// The device buffers a flattened program's job lists are uploaded to.
struct JobBufs {
    DevBuf *br, *ks, *fr, *sm, *tr;
};

uint64_t splitmix64(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Gate trace of one chunk of G gates: max(min(per_launch, G), ceil(G /
// one_in)) of them, chosen uniformly by the context's seeded generator, are
// copied after the chunk's key switch --
// their inputs are still intact then (a pool slot is rewritten only in a
// layer after its last reader) and their outputs are written.  Each record
// holds the gate's pre-combination with a multi-input sum expanded into its
// terms.
void trace_chunk(velopir_ctx *c, const Layer &L, const Chunk &ch, uint32_t *pool, const std::vector<int> &phys,
                 const std::unordered_map<uint64_t, const SumJob *> &sums, Flat &F)
{
    const size_t G = ch.g1 - ch.g0;
    size_t k = std::min<size_t>(G, c->trace_per_launch);
    if (c->trace_one_in) k = std::max(k, (G + c->trace_one_in - 1) / c->trace_one_in);
    if (k == 0 || c->trace_next >= c->trace_cap) return;
    std::vector<size_t> pick(k);
    for (size_t i = 0; i < G; ++i) {   // reservoir sampling of k of the G gates
        if (i < k) pick[i] = i;
        else if (size_t j = (size_t)(splitmix64(c->trace_rng) % (i + 1)); j < k) pick[j] = i;
    }
    std::sort(pick.begin(), pick.end());
    const size_t to = F.tr.size();
    for (size_t q : pick) {
        if (c->trace_next >= c->trace_cap) break;
        const KsJob &kj = L.ks[ch.g0 + q];
        TraceJob t{};
        bool ok = true;
        auto term = [&](int r, const uint32_t *p, int32_t sgn) {
            if (!p) return;
            const uint32_t *rp = resolve((uint64_t)(uintptr_t)p, pool, phys);
            int idx = -1;
            for (int m = 0; m < t.nin; ++m)
                if (t.in[m] == rp) idx = m;
            if (idx < 0) {
                if (t.nin == kSumMax) { ok = false; return; }
                idx = t.nin++;
                t.in[idx] = rp;
            }
            t.coef[r][idx] += sgn;
        };
        const int rot[2] = {kj.e0, kj.e1};
        for (int r = 0; r < 2 && rot[r] >= 0; ++r) {
            const BrJob &b = L.br[rot[r]];
            t.cst[r] = b.cst;
            t.nrot = r + 1;
            for (int w = 0; w < 2; ++w) {
                const uint32_t *in = w ? b.in1 : b.in0;
                const int32_t sgn = w ? b.s1 : b.s0;
                auto it = in ? sums.find((uint64_t)(uintptr_t)in) : sums.end();
                if (it != sums.end())
                    for (int m = 0; m < it->second->n; ++m) term(r, it->second->in[m], it->second->s[m] * sgn);
                else
                    term(r, in, sgn);
            }
        }
        if (!ok) continue;
        t.ks_cst = kj.cst;
        t.out = resolve((uint64_t)(uintptr_t)kj.out, pool, phys);
        t.rec = (int32_t)c->trace_next++;
        F.tr.push_back(t);
    }
    if (F.tr.size() > to) F.launches.push_back({4, to, (int)(F.tr.size() - to)});
}

// Append one layer's jobs: its multi-input sums first, then chunks whose
// blind rotations fit the extracted-row scratch (each followed by its key
// switch and, when tracing, its trace copies); pointers are resolved against
// `pool`.
void flatten_layer(velopir_ctx *c, const Layer &L, int cap, uint32_t *pool, const std::vector<int> &phys, Flat &F)
{
    std::unordered_map<uint64_t, const SumJob *> sums;
    if (!L.sm.empty()) {
        const size_t so = F.sm.size();
        for (const SumJob &x : L.sm) {
            SumJob sj = x;
            for (int k = 0; k < sj.n; ++k) sj.in[k] = resolve((uint64_t)(uintptr_t)sj.in[k], pool, phys);
            sj.out = resolve((uint64_t)(uintptr_t)sj.out, pool, phys);
            F.sm.push_back(sj);
            if (c->trace_on) sums[(uint64_t)(uintptr_t)x.out] = &x;
        }
        F.launches.push_back({3, so, (int)L.sm.size()});
    }
    std::vector<Chunk> chunks;
    layer_chunks(L, cap, chunks);
    for (const Chunk &ch : chunks) {
        const size_t bo = F.br.size();
        for (int b = ch.br0; b < ch.br1; ++b) {
            BrJob j = L.br[b];
            j.in0 = j.in0 ? resolve((uint64_t)(uintptr_t)j.in0, pool, phys) : nullptr;
            j.in1 = j.in1 ? resolve((uint64_t)(uintptr_t)j.in1, pool, phys) : nullptr;
            j.big = b - ch.br0;
            F.br.push_back(j);
        }
        F.launches.push_back({0, bo, ch.br1 - ch.br0});
        const size_t ko = F.ks.size();
        for (size_t q = ch.g0; q < ch.g1; ++q) {
            KsJob k = L.ks[q];
            k.e0 -= ch.br0;
            if (k.e1 >= 0) k.e1 -= ch.br0;
            k.out = resolve((uint64_t)(uintptr_t)k.out, pool, phys);
            F.ks.push_back(k);
        }
        F.launches.push_back({1, ko, (int)(ch.g1 - ch.g0)});
        if (c->trace_on) trace_chunk(c, L, ch, pool, phys, sums, F);
    }
}

void flatten_free(const std::vector<FreeJob> &fr, uint32_t *pool, const std::vector<int> &phys, Flat &F)
{
    if (fr.empty()) return;
    const size_t fo = F.fr.size();
    for (FreeJob f : fr) {
        f.in = f.in ? resolve((uint64_t)(uintptr_t)f.in, pool, phys) : nullptr;
        f.out = resolve((uint64_t)(uintptr_t)f.out, pool, phys);
        F.fr.push_back(f);
    }
    F.launches.push_back({2, fo, (int)fr.size()});
}

int ensure_path_key(velopir_ctx *c)
{
    if (!c->key_loaded) return fail(c, VELOPIR_ERR_NOKEY, "no cloud key loaded");
    if (c->path == VP_PATH_TENSOR_F16 && !c->bk_tc_ready) {
        int rc = ensure(c, c->bk_tc, bk_tc_bytes());
        if (rc) return rc;
        c->launches += prepare_bk_tc(as<uint32_t>(c->bk), c->bk_tc.p, c->stream);
        CU(cudaGetLastError());
        c->bk_tc_ready = true;
    }
    if (c->path == VP_PATH_NTT && !c->bk_ntt_ready) {
        int rc = ensure(c, c->bk_ntt, bk_ntt_words() * 4);
        if (rc) return rc;
        c->launches += prepare_bk_ntt(as<uint32_t>(c->bk), as<uint32_t>(c->bk_ntt), c->stream);
        CU(cudaGetLastError());
        c->bk_ntt_ready = true;
    }
    return VELOPIR_OK;
}

// Scratch of the tensor-core path for launches of up to `rows` bootstraps;
// sized before any launch is issued (and so before any stream capture).
int ensure_tc_scratch(velopir_ctx *c, int rows)
{
    return c->path == VP_PATH_TENSOR_F16 ? ensure(c, c->tc_scratch, tc_scratch_bytes(std::max(2, rows))) : VELOPIR_OK;
}

int launch_br(velopir_ctx *c, const BrJob *jobs, int n)
{
    if (c->path == VP_PATH_TENSOR_F16)
        return launch_br_tc(jobs, n, c->bk_tc.p, c->tc_scratch.p, as<uint32_t>(c->big), as<int>(c->errw), c->stream);
    if (c->path == VP_PATH_NTT)
        return launch_br_ntt(jobs, n, as<uint32_t>(c->bk_ntt), as<uint32_t>(c->big), as<int>(c->errw), c->stream);
    return launch_br_dense(jobs, n, as<uint32_t>(c->bk), as<uint32_t>(c->big), as<int>(c->errw), c->stream);
}

int upload(velopir_ctx *c, const Flat &F, const JobBufs &J)
{
    int rc;
    if ((rc = ensure(c, *J.br, std::max<size_t>(1, F.br.size()) * sizeof(BrJob)))) return rc;
    if ((rc = ensure(c, *J.ks, std::max<size_t>(1, F.ks.size()) * sizeof(KsJob)))) return rc;
    if ((rc = ensure(c, *J.fr, std::max<size_t>(1, F.fr.size()) * sizeof(FreeJob)))) return rc;
    if ((rc = ensure(c, *J.sm, std::max<size_t>(1, F.sm.size()) * sizeof(SumJob)))) return rc;
    if ((rc = ensure(c, *J.tr, std::max<size_t>(1, F.tr.size()) * sizeof(TraceJob)))) return rc;
    if (!F.br.empty()) CU(cudaMemcpyAsync(J.br->p, F.br.data(), F.br.size() * sizeof(BrJob), cudaMemcpyHostToDevice, c->stream));
    if (!F.ks.empty()) CU(cudaMemcpyAsync(J.ks->p, F.ks.data(), F.ks.size() * sizeof(KsJob), cudaMemcpyHostToDevice, c->stream));
    if (!F.fr.empty()) CU(cudaMemcpyAsync(J.fr->p, F.fr.data(), F.fr.size() * sizeof(FreeJob), cudaMemcpyHostToDevice, c->stream));
    if (!F.sm.empty()) CU(cudaMemcpyAsync(J.sm->p, F.sm.data(), F.sm.size() * sizeof(SumJob), cudaMemcpyHostToDevice, c->stream));
    if (!F.tr.empty()) CU(cudaMemcpyAsync(J.tr->p, F.tr.data(), F.tr.size() * sizeof(TraceJob), cudaMemcpyHostToDevice, c->stream));
    return VELOPIR_OK;
}

int launches_only(velopir_ctx *c, const Flat &F, const JobBufs &J);

JobBufs program_bufs(velopir_ctx *c) { return {&c->jobs_br, &c->jobs_ks, &c->jobs_fr, &c->jobs_sm, &c->jobs_tr}; }
JobBufs serving_bufs(velopir_ctx *c) { return {&c->s_br, &c->s_ks, &c->s_fr, &c->s_sm, &c->s_tr}; }

// Upload the flattened jobs and issue every launch in order.
int issue(velopir_ctx *c, const Flat &F, const JobBufs &J)
{
    int rc;
    if ((rc = upload(c, F, J))) return rc;
    return launches_only(c, F, J);
}

// The launch sequence captured once into a CUDA graph and replayed; the job
// lists are uploaded before each replay, so only the launch list (kinds,
// offsets, sizes) and the buffers must match the captured one.
int issue_graph(velopir_ctx *c, const Flat &F)
{
    int rc;
    const JobBufs J = program_bufs(c);
    if ((rc = upload(c, F, J))) return rc;
    std::vector<uint64_t> sig;
    sig.reserve(F.launches.size() * 3 + 12);
    for (const Launch &l : F.launches) {
        sig.push_back((uint64_t)l.kind);
        sig.push_back((uint64_t)l.off);
        sig.push_back((uint64_t)l.n);
    }
    for (const DevBuf *b : {J.br, J.ks, J.fr, J.sm, J.tr, &c->big, &c->bk, &c->bk_ntt, &c->ksk, &c->trace_buf,
                            &c->bk_tc, &c->tc_scratch})
        sig.push_back((uint64_t)(uintptr_t)b->p);
    sig.push_back((uint64_t)c->path);
    if (!c->graph_exec || sig != c->graph_sig) {
        if (c->graph_exec) {
            cudaGraphExecDestroy(c->graph_exec);
            c->graph_exec = nullptr;
        }
        const bool prof = c->prof;
        c->prof = false;
        cudaGraph_t g = nullptr;
        CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        rc = launches_only(c, F, J);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        c->prof = prof;
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return fail(c, VELOPIR_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(c, VELOPIR_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        c->graph_sig.swap(sig);
    } else {
        c->graph_replays++;
    }
    CU(cudaGraphLaunch(c->graph_exec, c->stream));
    return VELOPIR_OK;
}

int launches_only(velopir_ctx *c, const Flat &F, const JobBufs &J)
{
    // one NVTX range per launch (kind and size) for timeline tools
    static const char *names[5] = {"velopir:blind_rotate", "velopir:key_switch", "velopir:free_gates",
                                   "velopir:sum_precombine", "velopir:gate_trace"};
    for (const Launch &l : F.launches) {
        nvtxRangePushA(names[l.kind]);
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (c->prof) {
            for (cudaEvent_t *e : {&ea, &eb}) {
                if (!c->spare.empty()) { *e = c->spare.back(); c->spare.pop_back(); }
                else CU(cudaEventCreate(e));
            }
            CU(cudaEventRecord(ea, c->stream));
        }
        switch (l.kind) {
        case 0: c->launches += launch_br(c, as<BrJob>(*J.br) + l.off, l.n); break;
        case 1:
            c->launches += launch_key_switch(as<KsJob>(*J.ks) + l.off, l.n, as<uint32_t>(c->big), as<uint32_t>(c->ksk),
                                             as<int>(c->errw), c->stream);
            break;
        case 2: c->launches += launch_free(as<FreeJob>(*J.fr) + l.off, l.n, c->stream); break;
        case 3: c->launches += launch_sum(as<SumJob>(*J.sm) + l.off, l.n, c->stream); break;
        default: c->launches += launch_trace(as<TraceJob>(*J.tr) + l.off, l.n, as<uint32_t>(c->trace_buf), c->stream); break;
        }
        CU(cudaGetLastError());
        nvtxRangePop();
        if (c->prof) {
            CU(cudaEventRecord(eb, c->stream));
            c->recs.push_back({l.kind, (uint64_t)l.n, ea, eb});
        }
    }
    return VELOPIR_OK;
}

int prof_drain(velopir_ctx *c)
{
    if (c->recs.empty()) return VELOPIR_OK;
    CU(cudaStreamSynchronize(c->stream));
    for (auto &r : c->recs) {
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, r.a, r.b));
        c->prof_launches[r.kind] += 1;
        c->prof_units[r.kind] += r.units;
        c->prof_ms[r.kind] += ms;
        c->spare.push_back(r.a);
        c->spare.push_back(r.b);
    }
    c->recs.clear();
    return VELOPIR_OK;
}

int check_device_error(velopir_ctx *c)
{
    int h = 0;
    CU(cudaMemcpyAsync(&h, c->errw.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (h != kDevOk) {
        cudaMemsetAsync(c->errw.p, 0, sizeof(int), c->stream);
        return fail(c, VELOPIR_ERR_TIMEOUT, "a bounded device wait gave up (code %d)", h);
    }
    return VELOPIR_OK;
}

// Run a whole program synchronously with the context's shared scratch.
int run_program(velopir_ctx *c, Program &P, bool graph = false)
{
    int rc;
    if ((rc = ensure_path_key(c))) return rc;
    if (c->path == VP_PATH_NTT) relayer(P, ntt_full_wave());
    allocate_slots(P);
    if ((rc = ensure(c, c->pool, std::max<size_t>(1, (size_t)P.nphys) * kSlotWords * 4))) return rc;
    size_t max_br = 1;
    for (const Layer &L : P.layers) max_br = std::max(max_br, L.br.size());
    const int cap = chunk_capacity(max_br, c->big_rows);
    if ((rc = ensure(c, c->big, (size_t)std::max(2, cap) * kBigWords * 4))) return rc;
    if ((rc = ensure_tc_scratch(c, cap))) return rc;
    uint32_t *pool = as<uint32_t>(c->pool);
    Flat F;
    flatten_free(P.pre, pool, P.phys, F);
    for (const Layer &L : P.layers) {
        flatten_layer(c, L, cap, pool, P.phys, F);
        flatten_free(L.fr, pool, P.phys, F);
    }
    if (graph) rc = issue_graph(c, F);
    else rc = issue(c, F, program_bufs(c));
    if (rc) return rc;
    return check_device_error(c);
}

// Stage `words` uint32 of a caller buffer on the device (device pointers pass through).
int stage_in(velopir_ctx *c, const uint32_t *src, size_t words, size_t at_words, const uint32_t **dev)
{
    if (is_device_ptr(src)) {
        *dev = src;
        return VELOPIR_OK;
    }
    uint32_t *d = as<uint32_t>(c->in) + at_words;
    CU(cudaMemcpyAsync(d, src, words * 4, cudaMemcpyHostToDevice, c->stream));
    *dev = d;
    return VELOPIR_OK;
}

struct OutStage {
    uint32_t *user = nullptr;
    uint32_t *dev = nullptr;
    size_t words = 0;
    bool host = false;
};

int stage_out(velopir_ctx *c, uint32_t *user, size_t words, OutStage &o)
{
    o.user = user;
    o.words = words;
    o.host = !is_device_ptr(user);
    if (o.host) {
        int rc = ensure(c, c->out, std::max<size_t>(1, words) * 4);
        if (rc) return rc;
        o.dev = as<uint32_t>(c->out);
    } else {
        o.dev = user;
    }
    return VELOPIR_OK;
}

int finish_out(velopir_ctx *c, const OutStage &o)
{
    if (o.host && o.words) {
        CU(cudaMemcpyAsync(o.user, o.dev, o.words * 4, cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    return VELOPIR_OK;
}

bool params_ok(const velopir_params *p)
{
    return p && p->n == kn && p->N == kN && p->k == 1 && p->l == kL && p->bg_bits == kBgBits && p->ks_t == kKsT &&
           p->ks_base_bits == kKsBaseBits;
}

int build_batch(velopir_ctx *c, int gate, const uint32_t *din, uint32_t *dout, size_t count, Program &P)
{
    Builder B(P);
    const int ar = gate == G_MUX ? 3 : 2;
    for (size_t g = 0; g < count; ++g) {
        const uint32_t *base = din + g * ar * kLweWords;
        if (gate == G_MUX)
            B.mux(B.input(base), B.input(base + kLweWords), B.input(base + 2 * kLweWords), dout + g * kLweWords);
        else
            B.gate(gate, B.input(base), B.input(base + kLweWords), dout + g * kLweWords);
    }
    return VELOPIR_OK;
}

// ------------------------------ serving -----------------------------------

struct ServeQuery {
    uint64_t ticket = 0;
    velopir_query q{};
    std::vector<uint32_t> db, payload;   // host copies of the plaintext database
    Program P;
    size_t cursor = 0;      // next layer
    size_t offset = 0;      // gates of layer `cursor` already issued
    size_t sums_for = SIZE_MAX;   // layer whose multi-input sums were issued
    bool pre_done = false;
    size_t footprint = 0;
    uint32_t *dmem = nullptr;   // inputs + pool + output staging (one allocation)
    uint32_t *dout = nullptr;
    size_t out_words = 0;
    bool out_host = false;
    bool done = false;
    bool cancelled = false; // velopir_cancel: issue nothing more, report as cancelled
    cudaEvent_t ev = nullptr;
};

int agg_fanin(const velopir_query &q) { return q.agg_fanin >= 2 ? q.agg_fanin : 2; }

size_t query_in_words(const velopir_query &q)
{
    switch (q.kind) {
    case VP_QUERY_INTV: return 64 * (size_t)kLweWords;
    case VP_QUERY_COV: return 32 * (size_t)kLweWords;
    default: return (size_t)q.id_bits * kLweWords;
    }
}

size_t query_out_words(const velopir_query &q)
{
    if (q.kind == VP_QUERY_IDM && q.payload) return (size_t)q.payload_bits * kLweWords;
    return q.D * kLweWords;
}

int validate_query(velopir_ctx *c, const velopir_query &q)
{
    if (!q.enc_a || !q.out || (!q.db && q.D)) return fail(c, VELOPIR_ERR_ARG, "null query buffer");
    if (q.kind == VP_QUERY_INTV && !q.enc_b) return fail(c, VELOPIR_ERR_ARG, "IntV needs enc_b");
    if (q.kind < 0 || q.kind > 2) return fail(c, VELOPIR_ERR_ARG, "unknown query kind %d", q.kind);
    if (q.kind == VP_QUERY_IDM && (q.id_bits < 1 || q.id_bits > 32))
        return fail(c, VELOPIR_ERR_ARG, "id_bits must be in [1, 32]");
    if (q.kind == VP_QUERY_IDM && q.payload && (q.payload_bits < 1 || q.payload_bits > 32))
        return fail(c, VELOPIR_ERR_ARG, "payload_bits must be in [1, 32]");
    if (q.agg_fanin != 0 && (q.agg_fanin < 2 || q.agg_fanin > kMaxFanin))
        return fail(c, VELOPIR_ERR_ARG, "agg_fanin must be 0 or in [2, %d]", kMaxFanin);
    return VELOPIR_OK;
}

// Build the query's program against its own device block: [inputs | pool | out].
int build_query(velopir_ctx *c, ServeQuery &s)
{
    const velopir_query &q = s.q;
    const size_t inw = query_in_words(q);
    s.out_words = query_out_words(q);
    s.out_host = !is_device_ptr(q.out);
    // Build once with placeholder bases to learn the pool size, then rebuild.
    for (int pass = 0; pass < 2; ++pass) {
        s.P = Program();
        Builder B(s.P);
        // Pass 0 only sizes the pool: any non-null, untagged bases give the
        // same program shape as the real ones used in pass 1.
        uint32_t *in_base = pass == 0 ? reinterpret_cast<uint32_t *>(uintptr_t(1) << 20) : s.dmem;
        uint32_t *out_base = s.out_host ? (pass == 0 ? reinterpret_cast<uint32_t *>(uintptr_t(1) << 40) : s.dout)
                                        : q.out;
        std::vector<Ref> a(64), b(32);
        const int nin = (int)(inw / kLweWords);
        for (int i = 0; i < nin; ++i) a[i] = B.input(in_base + (size_t)i * kLweWords);
        if (q.kind == VP_QUERY_INTV)
            build_intv(B, a.data(), a.data() + 32, q.db, q.D, out_base);
        else if (q.kind == VP_QUERY_COV)
            build_cov(B, a.data(), q.db, q.D, out_base);
        else
            build_idm(B, a.data(), q.id_bits, q.db, q.D, q.payload, q.payload_bits, out_base, agg_fanin(q));
        if (c->path == VP_PATH_NTT) relayer(s.P, ntt_full_wave());
        allocate_slots(s.P);
        if (pass == 0) {
            s.footprint = (inw + (s.out_host ? s.out_words : 0) + (size_t)s.P.nphys * kSlotWords) * 4 + 256;
            if (c->budget && c->allocated + c->serve_reserved + s.footprint > c->budget) return VELOPIR_ERR_BUSY;
            void *p = nullptr;
            cudaError_t e = cudaMallocAsync(&p, s.footprint, c->stream);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return VELOPIR_ERR_BUSY;
            }
            s.dmem = reinterpret_cast<uint32_t *>(p);
            s.dout = s.dmem + inw;
            c->serve_reserved += s.footprint;
            // inputs
            CU(cudaMemcpyAsync(s.dmem, q.enc_a, (q.kind == VP_QUERY_INTV ? 32 : inw / kLweWords) * kLweWords * 4,
                               cudaMemcpyDefault, c->stream));
            if (q.kind == VP_QUERY_INTV)
                CU(cudaMemcpyAsync(s.dmem + 32 * kLweWords, q.enc_b, 32 * kLweWords * 4, cudaMemcpyDefault, c->stream));
        }
    }
    return VELOPIR_OK;
}

uint32_t *query_pool(const ServeQuery &s)
{
    return s.dmem + query_in_words(s.q) + (s.out_host ? s.out_words : 0);
}

// One serving step: the active queries contribute the gates of their current
// layers, oldest query first, up to a whole number of full waves of the
// blind-rotation kernel when at least one wave is available (else all of
// them); all of them run as one merged launch sequence.  A query whose layer
// is only partly issued continues it in the next step, so its layers still
// run in order.
int serve_step(velopir_ctx *c)
{
    int rc;
    // admit waiting queries while memory allows
    while (!c->waiting.empty()) {
        ServeQuery &s = *c->waiting.front();
        rc = build_query(c, s);
        if (rc == VELOPIR_ERR_BUSY) break;
        if (rc) return rc;
        c->active.push_back(std::move(c->waiting.front()));
        c->waiting.pop_front();
    }
    if (c->active.empty()) return VELOPIR_OK;
    if ((rc = ensure_path_key(c))) return rc;
    Flat F;
    // Each query's layer is chunked on its own; chunks of all queries are
    // concatenated per kind so one blind-rotation launch covers them all.
    Flat merged;
    size_t total_br = 0;
    for (auto &sp : c->active) {
        ServeQuery &s = *sp;
        if (!s.cancelled && s.cursor < s.P.layers.size()) {
            const Layer &L = s.P.layers[s.cursor];
            total_br += L.br.size() - (s.offset < L.ks.size() ? (size_t)L.ks[s.offset].e0 : L.br.size());
        }
    }
    const size_t wave = c->path == VP_PATH_NTT ? (size_t)ntt_full_wave() : 0;
    const size_t take = (wave && total_br >= wave) ? total_br / wave * wave : total_br;
    const int cap = chunk_capacity(take, c->big_rows);
    if ((rc = ensure(c, c->big, (size_t)std::max(2, cap) * kBigWords * 4))) return rc;
    if ((rc = ensure_tc_scratch(c, cap))) return rc;
    // Merge layer jobs of all queries into one virtual layer with rebased indices.
    Layer ML;
    std::vector<FreeJob> pre, post;
    for (auto &sp : c->active) {
        ServeQuery &s = *sp;
        uint32_t *pool = query_pool(s);
        if (!s.pre_done) {
            for (FreeJob f : s.P.pre) {
                f.in = f.in ? resolve((uint64_t)(uintptr_t)f.in, pool, s.P.phys) : nullptr;
                f.out = resolve((uint64_t)(uintptr_t)f.out, pool, s.P.phys);
                pre.push_back(f);
            }
            s.pre_done = true;
        }
        if (s.cancelled || s.cursor >= s.P.layers.size() || ML.br.size() >= take) continue;
        const Layer &L = s.P.layers[s.cursor];
        // the layer's multi-input sums run before the first of its rotations
        if (s.sums_for != s.cursor) {
            for (SumJob sj : L.sm) {
                for (int k = 0; k < sj.n; ++k) sj.in[k] = resolve((uint64_t)(uintptr_t)sj.in[k], pool, s.P.phys);
                sj.out = resolve((uint64_t)(uintptr_t)sj.out, pool, s.P.phys);
                ML.sm.push_back(sj);
            }
            s.sums_for = s.cursor;
        }
        // a gate's blind rotations are consecutive, in the order of its key switches
        for (; s.offset < L.ks.size(); ++s.offset) {
            KsJob k = L.ks[s.offset];
            const size_t nbr = k.e1 >= 0 ? 2 : 1;
            if (ML.br.size() + nbr > take && !ML.br.empty()) break;
            const int base = (int)ML.br.size();
            for (int e : {k.e0, k.e1}) {
                if (e < 0) continue;
                BrJob j = L.br[e];
                j.in0 = j.in0 ? resolve((uint64_t)(uintptr_t)j.in0, pool, s.P.phys) : nullptr;
                j.in1 = j.in1 ? resolve((uint64_t)(uintptr_t)j.in1, pool, s.P.phys) : nullptr;
                ML.br.push_back(j);
            }
            k.e0 = base;
            if (k.e1 >= 0) k.e1 = base + 1;
            k.out = resolve((uint64_t)(uintptr_t)k.out, pool, s.P.phys);
            ML.ks.push_back(k);
        }
        if (s.offset < L.ks.size()) continue;   // the rest of this layer goes in the next step
        for (FreeJob f : L.fr) {
            f.in = f.in ? resolve((uint64_t)(uintptr_t)f.in, pool, s.P.phys) : nullptr;
            f.out = resolve((uint64_t)(uintptr_t)f.out, pool, s.P.phys);
            post.push_back(f);
        }
        s.cursor++;
        s.offset = 0;
    }
    static const std::vector<int> nophys;
    flatten_free(pre, nullptr, nophys, merged);
    flatten_layer(c, ML, cap, nullptr, nophys, merged);
    flatten_free(post, nullptr, nophys, merged);
    if ((rc = issue(c, merged, serving_bufs(c)))) return rc;
    // completion bookkeeping
    for (auto &sp : c->active) {
        ServeQuery &s = *sp;
        if (s.cursor >= s.P.layers.size() && !s.ev) {
            if (s.out_host) CU(cudaMemcpyAsync(s.q.out, s.dout, s.out_words * 4, cudaMemcpyDeviceToHost, c->stream));
            CU(cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming));
            CU(cudaEventRecord(s.ev, c->stream));
        }
    }
    return VELOPIR_OK;
}

// Retire the admitted queries whose last work has finished.  sync_check
// reads the device error word synchronously; the issue thread checks it per
// step instead (without draining the stream).
int reap(velopir_ctx *c, bool sync_check = true)
{
    for (size_t i = 0; i < c->active.size();) {
        ServeQuery &s = *c->active[i];
        if (s.ev && cudaEventQuery(s.ev) == cudaSuccess) {
            int rc = sync_check ? check_device_error(c) : VELOPIR_OK;
            cudaEventDestroy(s.ev);
            s.ev = nullptr;
            cudaFreeAsync(s.dmem, c->stream);
            c->serve_reserved -= s.footprint;
            s.done = true;
            c->finished.push_back(std::move(c->active[i]));
            c->active.erase(c->active.begin() + i);
            if (rc) return rc;
        } else {
            ++i;
        }
    }
    return VELOPIR_OK;
}

// Whether any admitted query still has layers to issue.
bool issuable(const velopir_ctx *c)
{
    for (const auto &sp : c->active)
        if (!sp->cancelled && sp->cursor < sp->P.layers.size()) return true;
    return false;
}

constexpr int kMaxInflightSteps = 2;

// The issue thread: admits queries and issues serving steps back to back,
// keeping up to kMaxInflightSteps steps queued on the stream so that the GPU
// never waits for the host between steps.  After each step the error word is
// copied into a pinned slot; a bounded wait that gave up is reported once the
// step's event has completed.
void issue_loop(velopir_ctx *c)
{
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(c->mu);
    auto retire_front = [&]() {
        const velopir_ctx::Step st = c->inflight.front();
        c->inflight.pop_front();
        if (*st.err != kDevOk && c->issuer_rc == VELOPIR_OK) {
            c->issuer_rc = VELOPIR_ERR_TIMEOUT;
            c->issuer_err = "a bounded device wait gave up in a serving step";
            cudaMemsetAsync(c->errw.p, 0, sizeof(int), c->stream);
        }
        cudaEventDestroy(st.ev);
    };
    while (!c->stop_req) {
        while (!c->inflight.empty() && cudaEventQuery(c->inflight.front().ev) == cudaSuccess) retire_front();
        int rc = reap(c, false);
        if (rc && c->issuer_rc == VELOPIR_OK) { c->issuer_rc = rc; c->issuer_err = last_error_of(c); }
        if ((!c->waiting.empty() || issuable(c)) && (int)c->inflight.size() < kMaxInflightSteps &&
            c->issuer_rc == VELOPIR_OK) {
            rc = serve_step(c);
            if (rc != VELOPIR_OK) {
                c->issuer_rc = rc;
                c->issuer_err = last_error_of(c);
                continue;
            }
            // a slot of the pinned error copies that no in-flight step uses
            int *slot = c->err_host;
            for (int k = 0; k < kMaxInflightSteps; ++k) {
                bool used = false;
                for (const auto &st : c->inflight) used |= st.err == c->err_host + k;
                if (!used) { slot = c->err_host + k; break; }
            }
            cudaEvent_t ev = nullptr;
            if (cudaMemcpyAsync(slot, c->errw.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventRecord(ev, c->stream) != cudaSuccess) {
                c->issuer_rc = VELOPIR_ERR_CUDA;
                c->issuer_err = "serving step: event or copy failed";
                if (ev) cudaEventDestroy(ev);
                continue;
            }
            c->inflight.push_back({ev, slot});
            continue;
        }
        if (!c->inflight.empty()) {
            cudaEvent_t ev = c->inflight.front().ev;
            lk.unlock();
            cudaEventSynchronize(ev);
            lk.lock();
            continue;
        }
        bool pending = false;   // finished queries whose completion event is still outstanding
        for (const auto &sp : c->active) pending |= sp->ev != nullptr;
        lk.unlock();
        if (pending) std::this_thread::sleep_for(std::chrono::microseconds(200));
        else std::this_thread::sleep_for(std::chrono::milliseconds(1));
        lk.lock();
    }
    while (!c->inflight.empty()) {
        cudaEventSynchronize(c->inflight.front().ev);
        retire_front();
    }
    reap(c, false);
}

// Entry points other than the serving calls refuse to run while the issue
// thread owns the context's stream and scratch.
int busy(velopir_ctx *c)
{
    return c->serving ? fail(c, VELOPIR_ERR_BUSY, "the serving issue thread owns this context (velopir_serve_stop)")
                      : VELOPIR_OK;
}

}  // namespace

// Internal accessors for entry points defined in other translation units.
namespace vp {

int ctx_resources(velopir_ctx *c, CtxResources *r)
{
    if (!c || !r) return VELOPIR_ERR_ARG;
    if (int rc = busy(c)) return rc;
    r->device = c->device;
    r->stream = c->stream;
    r->key_loaded = c->key_loaded;
    r->bk = as<uint32_t>(c->bk);
    r->ksk = as<uint32_t>(c->ksk);
    r->bk_ntt = (c->path == VP_PATH_NTT && c->bk_ntt_ready) ? as<uint32_t>(c->bk_ntt) : nullptr;
    r->err = as<int>(c->errw);
    return VELOPIR_OK;
}

int ctx_fail(velopir_ctx *c, int code, const char *msg) { return fail(c, code, "%s", msg); }

int ctx_finish(velopir_ctx *c, uint64_t launches)
{
    c->launches += launches;
    CU(cudaGetLastError());
    return check_device_error(c);
}

}  // namespace vp

// ================================ C ABI ====================================

extern "C" {

int velopir_create(velopir_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream)
{
    velopir_ctx *c = nullptr;
    if (!out) return fail(c, VELOPIR_ERR_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(c, VELOPIR_ERR_NOCUDA, "no CUDA device visible");
    }
    if (device < 0 || device >= n) return fail(c, VELOPIR_ERR_ARG, "device %d out of range [0, %d)", device, n);
    if (cudaSetDevice(device) != cudaSuccess) return fail(c, VELOPIR_ERR_CUDA, "cudaSetDevice(%d) failed", device);
    std::unique_ptr<velopir_ctx> ctx(new velopir_ctx());
    c = ctx.get();
    c->device = device;
    c->budget = hbm_budget_bytes;
    if (cuda_stream) {
        c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    } else {
        CU(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    if (configure_br_dense() != 0 || configure_br_ntt() != 0 || configure_br_tc() != 0 || configure_key_switch() != 0)
        return fail(nullptr, VELOPIR_ERR_CUDA, "cannot raise the shared-memory limit of the blind-rotation kernels");
    int rc = ensure(c, c->errw, 256);
    if (rc) { g_create_error = last_error_of(c); return rc; }
    CU(cudaMemsetAsync(c->errw.p, 0, 256, c->stream));
    *out = ctx.release();
    return VELOPIR_OK;
}

int velopir_destroy(velopir_ctx *c)
{
    if (!c) return VELOPIR_OK;
    velopir_serve_stop(c);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto &s : c->active) {
        if (s->ev) cudaEventDestroy(s->ev);
        if (s->dmem) cudaFreeAsync(s->dmem, c->stream);
    }
    cudaStreamSynchronize(c->stream);
    DevBuf *bufs[] = {&c->bk, &c->ksk, &c->bk_ntt, &c->big, &c->jobs_br, &c->jobs_ks, &c->jobs_fr, &c->jobs_sm,
                      &c->jobs_tr, &c->pool, &c->in, &c->out, &c->errw, &c->s_br, &c->s_ks, &c->s_fr, &c->s_sm,
                      &c->s_tr, &c->trace_buf, &c->bk_tc, &c->tc_scratch};
    for (DevBuf *b : bufs) dev_free(c, *b);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    for (auto &r : c->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : c->spare) cudaEventDestroy(e);
    if (c->err_host) cudaFreeHost(c->err_host);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return VELOPIR_OK;
}

int velopir_load_cloud_key(velopir_ctx *c, const velopir_params *params, const uint32_t *bk, size_t bk_words,
                           const uint32_t *ksk, size_t ksk_words)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (!params_ok(params)) return fail(c, VELOPIR_ERR_ARG, "parameters must be n=630 N=1024 k=1 l=3 Bg=2^7 t=8 base=2^2");
    if (!bk || !ksk) return fail(c, VELOPIR_ERR_ARG, "null key buffer");
    if (bk_words != kBkWords) return fail(c, VELOPIR_ERR_ARG, "bk_words %zu != %zu", bk_words, kBkWords);
    if (ksk_words != kKskAbiWords) return fail(c, VELOPIR_ERR_ARG, "ksk_words %zu != %zu", ksk_words, kKskAbiWords);
    if (int rc = busy(c)) return rc;
    cudaSetDevice(c->device);
    int rc;
    if ((rc = ensure(c, c->bk, kBkWords * 4))) return rc;
    if ((rc = ensure(c, c->ksk, kKskDevWords * 4))) return rc;
    CU(cudaMemcpyAsync(c->bk.p, bk, kBkWords * 4, cudaMemcpyDefault, c->stream));
    // The ABI rows (631 words) are padded to 632 for 16-byte loads.
    if ((rc = ensure(c, c->in, kKskAbiWords * 4))) return rc;
    CU(cudaMemcpyAsync(c->in.p, ksk, kKskAbiWords * 4, cudaMemcpyDefault, c->stream));
    c->launches += launch_pad_ksk(as<uint32_t>(c->in), as<uint32_t>(c->ksk), c->stream);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(c->stream));
    c->key_loaded = true;
    c->bk_ntt_ready = false;
    c->bk_tc_ready = false;
    return VELOPIR_OK;
}

int velopir_set_path(velopir_ctx *c, velopir_path path)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (int rc = busy(c)) return rc;
    if (path != VP_PATH_INT32_DENSE && path != VP_PATH_NTT && path != VP_PATH_TENSOR_F16)
        return fail(c, VELOPIR_ERR_ARG, "path %d is not available in this build", (int)path);
    c->path = path;
    return VELOPIR_OK;
}

int velopir_set_launch_limit(velopir_ctx *c, size_t max_rotations)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (int rc = busy(c)) return rc;
    if (max_rotations > ((size_t)1 << 16)) return fail(c, VELOPIR_ERR_ARG, "max_rotations above 65536");
    c->big_rows = max_rotations ? (int)max_rotations : (1 << 16);
    return VELOPIR_OK;
}

int velopir_set_encdb_fanin(velopir_ctx *c, int fanin)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (int rc = busy(c)) return rc;
    if (fanin != 0 && (fanin < 2 || fanin > kMaxFanin))
        return fail(c, VELOPIR_ERR_ARG, "fanin must be 0 or in [2, %d]", kMaxFanin);
    c->enc_fanin = fanin ? fanin : 2;
    return VELOPIR_OK;
}

static int bootstrap_common(velopir_ctx *c, velopir_gate gate, const uint32_t *lwe_in, uint32_t *lwe_out,
                            size_t count, bool plain)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (int rc = busy(c)) return rc;
    if ((int)gate < VP_AND || (int)gate > VP_MUX) return fail(c, VELOPIR_ERR_ARG, "unknown gate %d", (int)gate);
    if (count == 0) return VELOPIR_OK;
    if (!lwe_in || !lwe_out) return fail(c, VELOPIR_ERR_ARG, "null ciphertext buffer");
    if (!c->key_loaded) return fail(c, VELOPIR_ERR_NOKEY, "no cloud key loaded");
    cudaSetDevice(c->device);
    const int ar = gate == VP_MUX ? 3 : 2;
    const size_t inw = count * ar * kLweWords;
    int rc;
    if (!is_device_ptr(lwe_in) && (rc = ensure(c, c->in, inw * 4))) return rc;
    const uint32_t *din = nullptr;
    if ((rc = stage_in(c, lwe_in, inw, 0, &din))) return rc;
    OutStage o;
    if ((rc = stage_out(c, lwe_out, count * kLweWords, o))) return rc;
    if (!plain) {
        Program P;
        build_batch(c, (int)gate, din, o.dev, count, P);
        if ((rc = run_program(c, P))) return rc;
    } else {
        for (size_t g = 0; g < count; ++g) {
            Program P;
            build_batch(c, (int)gate, din + g * ar * kLweWords, o.dev + g * kLweWords, 1, P);
            if ((rc = run_program(c, P))) return rc;
        }
    }
    return finish_out(c, o);
}

int velopir_bootstrap_batch(velopir_ctx *c, velopir_gate gate, const uint32_t *lwe_in, uint32_t *lwe_out, size_t count)
{
    return bootstrap_common(c, gate, lwe_in, lwe_out, count, false);
}

int velopir_bootstrap_plain(velopir_ctx *c, velopir_gate gate, const uint32_t *lwe_in, uint32_t *lwe_out, size_t count)
{
    return bootstrap_common(c, gate, lwe_in, lwe_out, count, true);
}

// The scheduler reads the plaintext database on the host: bring a
// device-resident database or payload over first.
static int host_plaintext(velopir_ctx *c, velopir_query &q, std::vector<uint32_t> &db, std::vector<uint32_t> &pay)
{
    const size_t dbw = q.kind == VP_QUERY_INTV ? 4 * q.D : q.D;
    if (q.db && q.D && is_device_ptr(q.db)) {
        db.resize(dbw);
        CU(cudaMemcpy(db.data(), q.db, dbw * 4, cudaMemcpyDeviceToHost));
        q.db = db.data();
    }
    if (q.payload && q.D && is_device_ptr(q.payload)) {
        pay.resize(q.D);
        CU(cudaMemcpy(pay.data(), q.payload, q.D * 4, cudaMemcpyDeviceToHost));
        q.payload = pay.data();
    }
    return VELOPIR_OK;
}

static int run_query(velopir_ctx *c, velopir_query q)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (int rc = busy(c)) return rc;
    int rc;
    if ((rc = validate_query(c, q))) return rc;
    std::vector<uint32_t> hdb, hpay;
    cudaSetDevice(c->device);
    if ((rc = host_plaintext(c, q, hdb, hpay))) return rc;
    if (!c->key_loaded) return fail(c, VELOPIR_ERR_NOKEY, "no cloud key loaded");
    cudaSetDevice(c->device);
    if (q.D == 0) return VELOPIR_OK;
    const size_t inw = query_in_words(q);
    if ((rc = ensure(c, c->in, inw * 4))) return rc;
    const uint32_t *din_a = nullptr, *din_b = nullptr;
    if (q.kind == VP_QUERY_INTV) {
        if ((rc = stage_in(c, q.enc_a, 32 * kLweWords, 0, &din_a))) return rc;
        if ((rc = stage_in(c, q.enc_b, 32 * kLweWords, 32 * kLweWords, &din_b))) return rc;
    } else {
        if ((rc = stage_in(c, q.enc_a, inw, 0, &din_a))) return rc;
    }
    OutStage o;
    if ((rc = stage_out(c, q.out, query_out_words(q), o))) return rc;
    Program P;
    Builder B(P);
    std::vector<Ref> a(32), b(32);
    const int na = q.kind == VP_QUERY_IDM ? q.id_bits : 32;
    for (int i = 0; i < na; ++i) a[i] = B.input(din_a + (size_t)i * kLweWords);
    if (q.kind == VP_QUERY_INTV)
        for (int i = 0; i < 32; ++i) b[i] = B.input(din_b + (size_t)i * kLweWords);
    if (q.kind == VP_QUERY_INTV) build_intv(B, a.data(), b.data(), q.db, q.D, o.dev);
    else if (q.kind == VP_QUERY_COV) build_cov(B, a.data(), q.db, q.D, o.dev);
    else build_idm(B, a.data(), q.id_bits, q.db, q.D, q.payload, q.payload_bits, o.dev, agg_fanin(q));
    if ((rc = run_program(c, P))) return rc;
    return finish_out(c, o);
}

int velopir_query_batch(velopir_ctx *c, const velopir_query *qs, size_t nq, int use_graph)
{
    if (!c || (!qs && nq)) return fail(c, VELOPIR_ERR_ARG, "null argument");
    if (int rc = busy(c)) return rc;
    if (!c->key_loaded) return fail(c, VELOPIR_ERR_NOKEY, "no cloud key loaded");
    cudaSetDevice(c->device);
    int rc;
    std::vector<velopir_query> q(qs, qs + nq);
    std::vector<std::vector<uint32_t>> hdb(nq), hpay(nq);
    size_t inw = 0, outw = 0;
    for (size_t i = 0; i < nq; ++i) {
        if ((rc = validate_query(c, q[i]))) return rc;
        if ((rc = host_plaintext(c, q[i], hdb[i], hpay[i]))) return rc;
        inw += query_in_words(q[i]);
        if (!is_device_ptr(q[i].out)) outw += query_out_words(q[i]);
    }
    if ((rc = ensure(c, c->in, std::max<size_t>(1, inw) * 4))) return rc;
    if ((rc = ensure(c, c->out, std::max<size_t>(1, outw) * 4))) return rc;
    Program P;
    Builder B(P);
    std::vector<OutStage> outs(nq);
    size_t ino = 0, outo = 0;
    for (size_t i = 0; i < nq; ++i) {
        const velopir_query &x = q[i];
        if (x.D == 0) continue;
        const uint32_t *da = nullptr, *db = nullptr;
        if (x.kind == VP_QUERY_INTV) {
            if ((rc = stage_in(c, x.enc_a, 32 * kLweWords, ino, &da))) return rc;
            if ((rc = stage_in(c, x.enc_b, 32 * kLweWords, ino + 32 * kLweWords, &db))) return rc;
        } else if ((rc = stage_in(c, x.enc_a, query_in_words(x), ino, &da))) {
            return rc;
        }
        ino += query_in_words(x);
        OutStage &o = outs[i];
        o.user = x.out;
        o.words = query_out_words(x);
        o.host = !is_device_ptr(x.out);
        o.dev = o.host ? as<uint32_t>(c->out) + outo : x.out;
        if (o.host) outo += o.words;
        std::vector<Ref> a(32), b(32);
        const int na = x.kind == VP_QUERY_IDM ? x.id_bits : 32;
        for (int k = 0; k < na; ++k) a[k] = B.input(da + (size_t)k * kLweWords);
        if (x.kind == VP_QUERY_INTV)
            for (int k = 0; k < 32; ++k) b[k] = B.input(db + (size_t)k * kLweWords);
        if (x.kind == VP_QUERY_INTV) build_intv(B, a.data(), b.data(), x.db, x.D, o.dev);
        else if (x.kind == VP_QUERY_COV) build_cov(B, a.data(), x.db, x.D, o.dev);
        else build_idm(B, a.data(), x.id_bits, x.db, x.D, x.payload, x.payload_bits, o.dev, agg_fanin(x));
    }
    if ((rc = run_program(c, P, use_graph != 0))) return rc;
    for (auto &o : outs)
        if (o.user && (rc = finish_out(c, o))) return rc;
    return VELOPIR_OK;
}

uint64_t velopir_graph_replays(velopir_ctx *c) { return c ? c->graph_replays : 0; }

int velopir_autotune(velopir_ctx *c, double *wave_ms_out, int n_out)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (int rc = busy(c)) return rc;
    cudaSetDevice(c->device);
    int rc;
    if ((rc = ensure_path_key(c))) return rc;
    if (c->path != VP_PATH_NTT) return VELOPIR_OK;   // the dense path has one shape
    int sms = 0;
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    const int nshapes = ntt_shape_count();
    const int njmax = sms * ntt_shape(nshapes - 1);
    if ((rc = ensure(c, c->big, (size_t)njmax * kBigWords * 4))) return rc;
    if ((rc = ensure(c, c->jobs_br, (size_t)njmax * sizeof(BrJob)))) return rc;
    // trivial inputs cost exactly as much as real ones: the kernels do not branch on data
    std::vector<BrJob> jobs(njmax);
    for (int j = 0; j < njmax; ++j) { jobs[j] = BrJob{}; jobs[j].big = j; }
    CU(cudaMemcpyAsync(c->jobs_br.p, jobs.data(), jobs.size() * sizeof(BrJob), cudaMemcpyHostToDevice, c->stream));
    cudaEvent_t a, b;
    CU(cudaEventCreate(&a));
    CU(cudaEventCreate(&b));
    for (int si = 0; si < nshapes; ++si) {
        const int w = ntt_shape(si);
        float best = 0;
        for (int rep = 0; rep < 3; ++rep) {
            CU(cudaEventRecord(a, c->stream));
            c->launches += launch_br_ntt_w(as<BrJob>(c->jobs_br), sms * w, as<uint32_t>(c->bk_ntt), as<uint32_t>(c->big),
                                           as<int>(c->errw), c->stream, w);
            CU(cudaEventRecord(b, c->stream));
            CU(cudaEventSynchronize(b));
            float ms = 0;
            CU(cudaEventElapsedTime(&ms, a, b));
            if (rep > 0 && (best == 0 || ms < best)) best = ms;   // rep 0 warms up
        }
        ntt_set_wave_ms(w, best);
        if (wave_ms_out && si < n_out) wave_ms_out[si] = best;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return check_device_error(c);
}

int velopir_tuned_shape(velopir_ctx *c, size_t count)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    return c->path == VP_PATH_NTT ? ntt_pick_warps((int)std::min<size_t>(count, 1u << 30)) : br_dense_jobs_per_cta();
}

// ---- encrypted database ----------------------------------------------------

extern "C++" {
namespace {

constexpr int kMaxEncPayloadBits = 4096;   // VELOPIR_MAX_ENC_PAYLOAD_BITS

// Stage the query and database ciphertexts (host or device) into the
// context's input scratch, run the program `build` makes, write the outputs.
template <typename F>
int run_encdb(velopir_ctx *c, const uint32_t *q0, size_t q0_cts, const uint32_t *q1, size_t q1_cts,
              const uint32_t *db0, size_t db0_cts, const uint32_t *db1, size_t db1_cts, uint32_t *out,
              size_t out_cts, F build)
{
    if (int rc = busy(c)) return rc;
    if (!c->key_loaded) return fail(c, VELOPIR_ERR_NOKEY, "no cloud key loaded");
    cudaSetDevice(c->device);
    int rc;
    const size_t w[4] = {q0_cts * kLweWords, q1_cts * kLweWords, db0_cts * kLweWords, db1_cts * kLweWords};
    if ((rc = ensure(c, c->in, std::max<size_t>(1, w[0] + w[1] + w[2] + w[3]) * 4))) return rc;
    const uint32_t *src[4] = {q0, q1, db0, db1}, *dev[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t at = 0;
    for (int i = 0; i < 4; ++i) {
        if (src[i] && w[i] && (rc = stage_in(c, src[i], w[i], at, &dev[i]))) return rc;
        at += w[i];
    }
    OutStage o;
    if ((rc = stage_out(c, out, out_cts * kLweWords, o))) return rc;
    Program P;
    Builder B(P);
    build(B, dev, o.dev);
    if ((rc = run_program(c, P))) return rc;
    return finish_out(c, o);
}

std::vector<Ref> inputs_of(Builder &B, const uint32_t *base, int count)
{
    std::vector<Ref> r(count);
    for (int i = 0; i < count; ++i) r[i] = B.input(base + (size_t)i * kLweWords);
    return r;
}

}  // namespace
}  // extern "C++"

int velopir_interval_query_encdb(velopir_ctx *c, const uint32_t *enc_x, const uint32_t *enc_y, int l,
                                 const uint32_t *enc_rects, size_t D, const uint32_t *enc_payload, int payload_bits,
                                 uint32_t *out)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (l < 1 || l > 32) return fail(c, VELOPIR_ERR_ARG, "l = %d is outside 1..32", l);
    if (enc_payload && (payload_bits < 1 || payload_bits > kMaxEncPayloadBits))
        return fail(c, VELOPIR_ERR_ARG, "payload_bits = %d is outside 1..%d", payload_bits, kMaxEncPayloadBits);
    if (D == 0) return VELOPIR_OK;
    if (!enc_x || !enc_y || !enc_rects || !out) return fail(c, VELOPIR_ERR_ARG, "null argument");
    const int pb = enc_payload ? payload_bits : 0;
    return run_encdb(c, enc_x, (size_t)l, enc_y, (size_t)l, enc_rects, D * 4 * (size_t)l, enc_payload,
                     D * (size_t)pb, out, enc_payload ? (size_t)pb : D,
                     [&](Builder &B, const uint32_t *const *dev, uint32_t *o) {
                         const std::vector<Ref> x = inputs_of(B, dev[0], l), y = inputs_of(B, dev[1], l);
                         build_intv_enc(B, x.data(), y.data(), l, dev[2], D, dev[3], pb, o, c->enc_fanin);
                     });
}

int velopir_coordinate_query_encdb(velopir_ctx *c, const uint32_t *enc_cell, int w, const uint32_t *enc_cells,
                                   size_t D, const uint32_t *enc_payload, int payload_bits, uint32_t *out)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (w < 1 || w > 16) return fail(c, VELOPIR_ERR_ARG, "w = %d is outside 1..16", w);
    if (enc_payload && (payload_bits < 1 || payload_bits > kMaxEncPayloadBits))
        return fail(c, VELOPIR_ERR_ARG, "payload_bits = %d is outside 1..%d", payload_bits, kMaxEncPayloadBits);
    if (D == 0) return VELOPIR_OK;
    if (!enc_cell || !enc_cells || !out) return fail(c, VELOPIR_ERR_ARG, "null argument");
    const int pb = enc_payload ? payload_bits : 0;
    return run_encdb(c, enc_cell, 2 * (size_t)w, nullptr, 0, enc_cells, D * 2 * (size_t)w, enc_payload,
                     D * (size_t)pb, out, enc_payload ? (size_t)pb : D,
                     [&](Builder &B, const uint32_t *const *dev, uint32_t *o) {
                         const std::vector<Ref> cell = inputs_of(B, dev[0], 2 * w);
                         build_cov_enc(B, cell.data(), w, dev[2], D, dev[3], pb, o, c->enc_fanin);
                     });
}

int velopir_id_match_encdb(velopir_ctx *c, const uint32_t *enc_id, int id_bits, const uint32_t *enc_ids, size_t D,
                           const uint32_t *enc_payload, int payload_bits, uint32_t *out)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (id_bits < 1 || id_bits > 32) return fail(c, VELOPIR_ERR_ARG, "id_bits = %d is outside 1..32", id_bits);
    if (enc_payload && (payload_bits < 1 || payload_bits > kMaxEncPayloadBits))
        return fail(c, VELOPIR_ERR_ARG, "payload_bits = %d is outside 1..%d", payload_bits, kMaxEncPayloadBits);
    if (D == 0) return VELOPIR_OK;
    if (!enc_id || !enc_ids || !out) return fail(c, VELOPIR_ERR_ARG, "null argument");
    const int pb = enc_payload ? payload_bits : 0;
    return run_encdb(c, enc_id, (size_t)id_bits, nullptr, 0, enc_ids, D * (size_t)id_bits, enc_payload,
                     D * (size_t)pb, out, enc_payload ? (size_t)pb : D,
                     [&](Builder &B, const uint32_t *const *dev, uint32_t *o) {
                         const std::vector<Ref> id = inputs_of(B, dev[0], id_bits);
                         build_idm_enc(B, id.data(), id_bits, dev[2], D, dev[3], pb, o, c->enc_fanin);
                     });
}

int velopir_interval_query(velopir_ctx *c, const uint32_t *enc_x, const uint32_t *enc_y, const uint32_t *rects,
                           size_t D, uint32_t *out_bits)
{
    velopir_query q{};
    q.kind = VP_QUERY_INTV;
    q.enc_a = enc_x;
    q.enc_b = enc_y;
    q.db = rects;
    q.D = D;
    q.out = out_bits;
    return run_query(c, q);
}

int velopir_coordinate_query(velopir_ctx *c, const uint32_t *enc_cell, const uint32_t *cells, size_t D,
                             uint32_t *out_bits)
{
    velopir_query q{};
    q.kind = VP_QUERY_COV;
    q.enc_a = enc_cell;
    q.db = cells;
    q.D = D;
    q.out = out_bits;
    return run_query(c, q);
}

int velopir_id_match(velopir_ctx *c, const uint32_t *enc_id, int id_bits, const uint32_t *ids, size_t D,
                     const uint32_t *payload, int payload_bits, uint32_t *out)
{
    velopir_query q{};
    q.kind = VP_QUERY_IDM;
    q.id_bits = id_bits;
    q.payload_bits = payload ? payload_bits : 0;
    q.enc_a = enc_id;
    q.db = ids;
    q.payload = payload;
    q.D = D;
    q.out = out;
    return run_query(c, q);
}

int velopir_submit(velopir_ctx *c, const velopir_query *q, uint64_t *ticket)
{
    if (!c || !q || !ticket) return fail(c, VELOPIR_ERR_ARG, "null argument");
    int rc;
    if ((rc = validate_query(c, *q))) return rc;
    if (!c->key_loaded) return fail(c, VELOPIR_ERR_NOKEY, "no cloud key loaded");
    if (q->D == 0) return fail(c, VELOPIR_ERR_ARG, "empty database");
    if (c->waiting.size() >= 4096) return fail(c, VELOPIR_ERR_BUSY, "serving queue full");
    std::unique_ptr<ServeQuery> s(new ServeQuery());
    s->q = *q;
    cudaSetDevice(c->device);
    {
        const size_t dbw = q->kind == VP_QUERY_INTV ? 4 * q->D : q->D;
        s->db.resize(dbw);
        CU(cudaMemcpy(s->db.data(), q->db, dbw * 4, cudaMemcpyDefault));
        s->q.db = s->db.data();
        if (q->payload) {
            s->payload.resize(q->D);
            CU(cudaMemcpy(s->payload.data(), q->payload, q->D * 4, cudaMemcpyDefault));
            s->q.payload = s->payload.data();
        }
    }
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->waiting.size() >= 4096) return fail(c, VELOPIR_ERR_BUSY, "serving queue full");
    s->ticket = c->next_ticket++;
    *ticket = s->ticket;
    c->waiting.push_back(std::move(s));
    return VELOPIR_OK;
}

int velopir_cancel(velopir_ctx *c, uint64_t ticket)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    for (auto it = c->waiting.begin(); it != c->waiting.end(); ++it)
        if ((*it)->ticket == ticket) {   // never admitted: nothing on the device
            (*it)->cancelled = true;
            c->finished.push_back(std::move(*it));
            c->waiting.erase(it);
            return VELOPIR_OK;
        }
    for (auto &s : c->active)
        if (s->ticket == ticket) {
            if (!s->ev) {   // marks the end of the work already issued for it
                s->cancelled = true;
                CU(cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming));
                CU(cudaEventRecord(s->ev, c->stream));
            }
            return VELOPIR_OK;   // finishing already (its last layer is issued): it completes normally
        }
    for (auto &s : c->finished)
        if (s->ticket == ticket) return VELOPIR_OK;
    return fail(c, VELOPIR_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
}

int velopir_poll(velopir_ctx *c, uint64_t ticket, int *done)
{
    if (!c || !done) return fail(c, VELOPIR_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    *done = 0;
    if (c->serving && c->issuer_rc != VELOPIR_OK) return fail(c, c->issuer_rc, "%s", c->issuer_err.c_str());
    for (auto it = c->finished.begin(); it != c->finished.end(); ++it)
        if ((*it)->ticket == ticket) {
            *done = 1;
            const bool cancelled = (*it)->cancelled;
            c->finished.erase(it);
            if (cancelled) return fail(c, VELOPIR_ERR_CANCELLED, "ticket %llu was cancelled", (unsigned long long)ticket);
            return VELOPIR_OK;
        }
    bool known = false;
    for (auto &s : c->active) known |= s->ticket == ticket;
    for (auto &s : c->waiting) known |= s->ticket == ticket;
    if (!known) return fail(c, VELOPIR_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    if (c->serving) return VELOPIR_OK;   // the issue thread steps the loop
    int rc = serve_step(c);
    if (rc) return rc;
    // keep at most one step in flight ahead of the host
    for (auto &s : c->active)
        if (s->ev) cudaEventSynchronize(s->ev);
    if ((rc = reap(c))) return rc;
    for (auto it = c->finished.begin(); it != c->finished.end(); ++it)
        if ((*it)->ticket == ticket) {
            *done = 1;
            const bool cancelled = (*it)->cancelled;
            c->finished.erase(it);
            if (cancelled) return fail(c, VELOPIR_ERR_CANCELLED, "ticket %llu was cancelled", (unsigned long long)ticket);
            break;
        }
    return VELOPIR_OK;
}

int velopir_progress(velopir_ctx *c, uint64_t *done, size_t cap, size_t *ndone)
{
    if (!c || !ndone || (!done && cap)) return fail(c, VELOPIR_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    *ndone = 0;
    int rc;
    if (c->serving && c->issuer_rc != VELOPIR_OK) return fail(c, c->issuer_rc, "%s", c->issuer_err.c_str());
    if (!c->serving && (!c->waiting.empty() || !c->active.empty())) {
        if ((rc = serve_step(c))) return rc;
        for (auto &s : c->active)
            if (s->ev) cudaEventSynchronize(s->ev);
        if ((rc = reap(c))) return rc;
    }
    while (!c->finished.empty() && *ndone < cap) {
        done[(*ndone)++] = c->finished.front()->ticket;
        c->finished.erase(c->finished.begin());
    }
    return VELOPIR_OK;
}

int velopir_queue_depth(velopir_ctx *c, size_t *admitted, size_t *waiting)
{
    if (!c || !admitted || !waiting) return fail(c, VELOPIR_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(c->mu);
    *admitted = c->active.size();
    *waiting = c->waiting.size();
    return VELOPIR_OK;
}

int velopir_serve_start(velopir_ctx *c)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (c->serving) return VELOPIR_OK;
    if (!c->key_loaded) return fail(c, VELOPIR_ERR_NOKEY, "no cloud key loaded");
    cudaSetDevice(c->device);
    int rc;
    if ((rc = ensure_path_key(c))) return rc;
    if (!c->err_host) CU(cudaMallocHost(&c->err_host, kMaxInflightSteps * sizeof(int)));
    std::lock_guard<std::mutex> lk(c->mu);
    c->stop_req = false;
    c->issuer_rc = VELOPIR_OK;
    c->issuer_err.clear();
    c->serving = true;
    c->issuer = std::thread(issue_loop, c);
    return VELOPIR_OK;
}

int velopir_serve_stop(velopir_ctx *c)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (!c->serving) return VELOPIR_OK;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->stop_req = true;
    }
    c->issuer.join();
    c->serving = false;
    const int rc = c->issuer_rc;
    c->issuer_rc = VELOPIR_OK;
    if (rc != VELOPIR_OK) return fail(c, rc, "%s", c->issuer_err.c_str());
    return VELOPIR_OK;
}

int velopir_sync(velopir_ctx *c)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (int rc = busy(c)) return rc;
    cudaSetDevice(c->device);
    CU(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

const char *velopir_last_error(velopir_ctx *c)
{
    if (!c) return g_create_error.c_str();
    thread_local std::string copy;   // stable for the caller while another thread may fail
    copy = last_error_of(c);
    return copy.c_str();
}

uint64_t velopir_launch_count(velopir_ctx *c) { return c ? c->launches : 0; }

int velopir_selftest_wait_timeout(velopir_ctx *c)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (int rc = busy(c)) return rc;
    cudaSetDevice(c->device);
    c->launches += launch_wait_selftest(as<int>(c->errw), c->stream);
    CU(cudaGetLastError());
    return check_device_error(c);
}

int velopir_trace_start(velopir_ctx *c, uint64_t seed, uint32_t per_launch, uint32_t one_in, size_t cap)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (int rc = busy(c)) return rc;
    if ((per_launch == 0 && one_in == 0) || cap == 0 || cap > ((size_t)1 << 20))
        return fail(c, VELOPIR_ERR_ARG, "per_launch or one_in must be >= 1, and cap in [1, 2^20]");
    cudaSetDevice(c->device);
    const size_t bytes = cap * (size_t)kTraceWords * 4;
    int rc;
    if ((rc = ensure(c, c->trace_buf, bytes))) return rc;
    CU(cudaMemsetAsync(c->trace_buf.p, 0, bytes, c->stream));
    c->trace_on = true;
    c->trace_rng = seed;
    c->trace_per_launch = per_launch;
    c->trace_one_in = one_in;
    c->trace_cap = cap;
    c->trace_next = 0;
    return VELOPIR_OK;
}

int velopir_trace_stop(velopir_ctx *c, velopir_trace_rec *out, size_t cap, size_t *count)
{
    if (!c || !count || (!out && cap)) return fail(c, VELOPIR_ERR_ARG, "null argument");
    if (int rc = busy(c)) return rc;
    cudaSetDevice(c->device);
    *count = c->trace_on ? c->trace_next : 0;
    if (c->trace_on) {
        const size_t n = std::min(cap, c->trace_next);
        if (n) CU(cudaMemcpyAsync(out, c->trace_buf.p, n * sizeof(velopir_trace_rec), cudaMemcpyDefault, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    c->trace_on = false;
    dev_free(c, c->trace_buf);
    return check_device_error(c);
}

int velopir_profile(velopir_ctx *c, int enable)
{
    if (!c) return fail(c, VELOPIR_ERR_ARG, "ctx is NULL");
    if (int rc = busy(c)) return rc;
    cudaSetDevice(c->device);
    int rc = prof_drain(c);
    if (rc) return rc;
    for (int k = 0; k < 5; ++k) { c->prof_launches[k] = c->prof_units[k] = 0; c->prof_ms[k] = 0; }
    c->prof = enable != 0;
    return VELOPIR_OK;
}

int velopir_profile_read(velopir_ctx *c, int kernel, uint64_t *launches, uint64_t *units, double *ms)
{
    if (!c || kernel < 0 || kernel > 4 || !launches || !units || !ms) return fail(c, VELOPIR_ERR_ARG, "bad argument");
    if (int rc = busy(c)) return rc;
    cudaSetDevice(c->device);
    int rc = prof_drain(c);
    if (rc) return rc;
    *launches = c->prof_launches[kernel];
    *units = c->prof_units[kernel];
    *ms = c->prof_ms[kernel];
    return VELOPIR_OK;
}

}  // extern "C"
