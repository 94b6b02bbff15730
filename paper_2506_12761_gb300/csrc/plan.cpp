// Host-only dry run of a query's launch plan (velopir_plan_query in
// include/velopir.h).  It builds the same gate program as the device path,
// schedules it with the same list scheduler and slot allocator, and executes
// the result on noiseless plaintext phases: every stored ciphertext becomes
// its message +-1/8 (Section 2.2 Ecd), a blind rotation + extraction the sign
// of its pre-combined phase (phase 0 decodes as true, as the test vector
// X^{-bbar} v gives), and key switching and free gates the same mod-2^32 sums
// as on the device.  Each physical pool slot remembers which value it holds,
// so a read of a value that is not yet written, or already overwritten, is
// reported instead of silently computed.
#include <unordered_map>
#include <vector>

#include "../../include/velopir.h"
#include "sched.h"

using namespace vp;

namespace {

size_t plan_in_bits(const velopir_query &q) { return q.kind == VP_QUERY_IDM ? (size_t)q.id_bits : 32; }

size_t plan_out_bits(const velopir_query &q)
{
    return (q.kind == VP_QUERY_IDM && q.payload) ? (size_t)q.payload_bits : q.D;
}

struct Exec {
    const Program &P;
    std::unordered_map<uint64_t, uint32_t> mem;   // device addresses written so far
    std::vector<uint32_t> pool;
    std::vector<int> owner;                       // virtual slot held by each physical slot
    bool bad = false;

    explicit Exec(const Program &p) : P(p), pool(p.nphys, 0u), owner(p.nphys, -1) {}

    uint32_t read(const void *a)
    {
        const uint64_t v = (uint64_t)(uintptr_t)a;
        if (!v) return 0u;
        if (v & kSlotTag) {
            const int s = (int)(v & ~kSlotTag), ph = P.phys[s];
            if (owner[ph] != s) bad = true;
            return pool[ph];
        }
        auto it = mem.find(v);
        if (it == mem.end()) {
            bad = true;
            return 0u;
        }
        return it->second;
    }

    void write(const void *a, uint32_t x)
    {
        const uint64_t v = (uint64_t)(uintptr_t)a;
        if (v & kSlotTag) {
            const int s = (int)(v & ~kSlotTag), ph = P.phys[s];
            owner[ph] = s;
            pool[ph] = x;
        } else {
            mem[v] = x;
        }
    }

    void free_jobs(const std::vector<FreeJob> &fr)
    {
        for (const FreeJob &f : fr) write(f.out, (uint32_t)f.s * read(f.in) + f.cst);
    }
};

}  // namespace

extern "C" int velopir_plan_query(const velopir_query *q, int wave, const uint32_t *bits_a, const uint32_t *bits_b,
                                  uint32_t *bits_out, size_t *launch_sizes, int max_launches)
{
    if (!q || !q->db || q->D == 0 || !bits_a || !bits_out || wave < 0) return VELOPIR_ERR_ARG;
    if (q->kind != VP_QUERY_INTV && q->kind != VP_QUERY_COV && q->kind != VP_QUERY_IDM) return VELOPIR_ERR_ARG;
    if (q->kind == VP_QUERY_INTV && !bits_b) return VELOPIR_ERR_ARG;
    if (q->kind == VP_QUERY_IDM && (q->id_bits < 1 || q->id_bits > 32)) return VELOPIR_ERR_ARG;
    if (q->kind == VP_QUERY_IDM && q->payload && (q->payload_bits < 1 || q->payload_bits > 32)) return VELOPIR_ERR_ARG;
    if (launch_sizes && max_launches < 0) return VELOPIR_ERR_ARG;

    // stand-in device addresses: distinct, 16-byte aligned, never dereferenced
    uint32_t *in_a = reinterpret_cast<uint32_t *>(uintptr_t(1) << 32);
    uint32_t *in_b = reinterpret_cast<uint32_t *>(uintptr_t(2) << 32);
    uint32_t *out = reinterpret_cast<uint32_t *>(uintptr_t(3) << 32);
    Program P;
    Builder B(P);
    const size_t na = plan_in_bits(*q);
    std::vector<Ref> a(32), b(32);
    for (size_t i = 0; i < na; ++i) a[i] = B.input(in_a + i * kLweWords);
    if (q->kind == VP_QUERY_INTV)
        for (size_t i = 0; i < 32; ++i) b[i] = B.input(in_b + i * kLweWords);
    if (q->kind == VP_QUERY_INTV) build_intv(B, a.data(), b.data(), q->db, q->D, out);
    else if (q->kind == VP_QUERY_COV) build_cov(B, a.data(), q->db, q->D, out);
    else build_idm(B, a.data(), q->id_bits, q->db, q->D, q->payload, q->payload_bits, out);
    relayer(P, wave);
    allocate_slots(P);

    Exec X(P);
    auto enc = [](uint32_t bit) { return bit ? kMu : 0u - kMu; };
    for (size_t i = 0; i < na; ++i) X.write(in_a + i * kLweWords, enc(bits_a[i] & 1u));
    if (q->kind == VP_QUERY_INTV)
        for (size_t i = 0; i < 32; ++i) X.write(in_b + i * kLweWords, enc(bits_b[i] & 1u));
    X.free_jobs(P.pre);
    std::vector<uint32_t> ext;
    for (size_t l = 0; l < P.layers.size(); ++l) {
        const Layer &L = P.layers[l];
        // every blind rotation of a launch reads before any key switch writes
        ext.resize(L.br.size());
        for (size_t r = 0; r < L.br.size(); ++r) {
            const BrJob &j = L.br[r];
            const uint32_t c = j.cst + (uint32_t)j.s0 * X.read(j.in0) + (uint32_t)j.s1 * X.read(j.in1);
            ext[r] = (int32_t)c >= 0 ? kMu : 0u - kMu;
        }
        for (const KsJob &k : L.ks) X.write(k.out, ext[k.e0] + (k.e1 >= 0 ? ext[k.e1] : 0u) + k.cst);
        X.free_jobs(L.fr);
        if (launch_sizes && (int)l < max_launches) launch_sizes[l] = L.br.size();
    }
    const size_t nout = plan_out_bits(*q);
    for (size_t i = 0; i < nout; ++i) bits_out[i] = (int32_t)X.read(out + i * kLweWords) >= 0 ? 1u : 0u;
    if (X.bad) return VELOPIR_ERR_PLAN;
    return (int)P.layers.size();
}
