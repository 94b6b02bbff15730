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
#include <algorithm>
#include <unordered_map>
#include <vector>

#include "../../include/velopir.h"
#include "sched.h"

using namespace vp;

namespace {

size_t plan_out_bits(const velopir_query &q)
{
    return q.payload ? (size_t)q.payload_bits : q.D;
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

// Execute a scheduled program in the device's launch order: a layer's
// multi-input sums first, then its gates in the executor's chunks (the shared
// layer_chunks for a scratch of chunk_rows rows, clamped as the executor
// clamps it; 0: one chunk per layer), every chunk's blind rotations reading
// before its key switches write.  launch_sizes[l] receives the blind
// rotations of layer l.
void execute(const Program &P, Exec &X, int chunk_rows, size_t *launch_sizes, int max_launches)
{
    X.free_jobs(P.pre);
    size_t max_br = 1;
    for (const Layer &L : P.layers) max_br = std::max(max_br, L.br.size());
    const int cap = chunk_rows > 0 ? chunk_capacity(max_br, chunk_rows) : 0;
    std::vector<uint32_t> ext;
    std::vector<Chunk> chunks;
    for (size_t l = 0; l < P.layers.size(); ++l) {
        const Layer &L = P.layers[l];
        for (const SumJob &sj : L.sm) {
            uint32_t v = 0u;
            for (int k = 0; k < sj.n; ++k) v += (uint32_t)sj.s[k] * X.read(sj.in[k]);
            X.write(sj.out, v);
        }
        layer_chunks(L, cap, chunks);
        for (const Chunk &ch : chunks) {
            ext.assign((size_t)(ch.br1 - ch.br0), 0u);
            for (int r = ch.br0; r < ch.br1; ++r) {
                const BrJob &j = L.br[r];
                const uint32_t c = j.cst + (uint32_t)j.s0 * X.read(j.in0) + (uint32_t)j.s1 * X.read(j.in1);
                ext[r - ch.br0] = (int32_t)c >= 0 ? kMu : 0u - kMu;
            }
            for (size_t q = ch.g0; q < ch.g1; ++q) {
                const KsJob &k = L.ks[q];
                X.write(k.out, ext[k.e0 - ch.br0] + (k.e1 >= 0 ? ext[k.e1 - ch.br0] : 0u) + k.cst);
            }
        }
        X.free_jobs(L.fr);
        if (launch_sizes && (int)l < max_launches) launch_sizes[l] = L.br.size();
    }
}

bool plain_kind_ok(const velopir_query &q)
{
    if (!q.db || q.D == 0) return false;
    if (q.kind != VP_QUERY_INTV && q.kind != VP_QUERY_COV && q.kind != VP_QUERY_IDM) return false;
    if (q.kind == VP_QUERY_IDM && (q.id_bits < 1 || q.id_bits > 32)) return false;
    if (q.payload && (q.kind != VP_QUERY_IDM || q.payload_bits < 1 || q.payload_bits > 32)) return false;
    if (q.agg_fanin != 0 && (q.agg_fanin < 2 || q.agg_fanin > kMaxFanin)) return false;
    return true;
}

}  // namespace

extern "C" int velopir_plan_batch(const velopir_query *qs, size_t nq, int wave, int chunk_rows, const uint32_t *bits_a,
                                  const uint32_t *bits_b, uint32_t *bits_out, size_t *launch_sizes, int max_launches)
{
    if (!qs || !nq || !bits_a || !bits_out || wave < 0 || chunk_rows < 0) return VELOPIR_ERR_ARG;
    if (launch_sizes && max_launches < 0) return VELOPIR_ERR_ARG;
    for (size_t i = 0; i < nq; ++i) {
        if (!plain_kind_ok(qs[i])) return VELOPIR_ERR_ARG;
        if (qs[i].kind == VP_QUERY_INTV && !bits_b) return VELOPIR_ERR_ARG;
    }
    // stand-in device addresses: each query's inputs and outputs in regions of their own
    const uintptr_t in_base = uintptr_t(1) << 36, out_base = uintptr_t(2) << 36;
    Program P;
    Builder B(P);
    std::vector<std::pair<uint32_t *, uint32_t>> inputs;   // address, bit
    std::vector<uint32_t *> outs;
    size_t ia = 0, ib = 0, ino = 0, outo = 0;
    for (size_t i = 0; i < nq; ++i) {
        const velopir_query &q = qs[i];
        const size_t na = q.kind == VP_QUERY_IDM ? (size_t)q.id_bits : 32;
        const size_t nb = q.kind == VP_QUERY_INTV ? 32 : 0;
        uint32_t *in = reinterpret_cast<uint32_t *>(in_base) + ino;
        uint32_t *out = reinterpret_cast<uint32_t *>(out_base) + outo;
        std::vector<Ref> a(na), b(nb);
        for (size_t k = 0; k < na; ++k) {
            a[k] = B.input(in + k * kLweWords);
            inputs.emplace_back(in + k * kLweWords, bits_a[ia++] & 1u);
        }
        for (size_t k = 0; k < nb; ++k) {
            b[k] = B.input(in + (na + k) * kLweWords);
            inputs.emplace_back(in + (na + k) * kLweWords, bits_b[ib++] & 1u);
        }
        if (q.kind == VP_QUERY_INTV) build_intv(B, a.data(), b.data(), q.db, q.D, out);
        else if (q.kind == VP_QUERY_COV) build_cov(B, a.data(), q.db, q.D, out);
        else build_idm(B, a.data(), q.id_bits, q.db, q.D, q.payload, q.payload_bits, out,
                       q.agg_fanin >= 2 ? q.agg_fanin : 2);
        const size_t nout = plan_out_bits(q);
        for (size_t k = 0; k < nout; ++k) outs.push_back(out + k * kLweWords);
        ino += (na + nb) * kLweWords;
        outo += nout * kLweWords;
    }
    relayer(P, wave);
    allocate_slots(P);
    Exec X(P);
    for (auto &w : inputs) X.write(w.first, w.second ? kMu : 0u - kMu);
    execute(P, X, chunk_rows, launch_sizes, max_launches);
    for (size_t k = 0; k < outs.size(); ++k) bits_out[k] = (int32_t)X.read(outs[k]) >= 0 ? 1u : 0u;
    if (X.bad) return VELOPIR_ERR_PLAN;
    return (int)P.layers.size();
}

extern "C" int velopir_plan_query(const velopir_query *q, int wave, const uint32_t *bits_a, const uint32_t *bits_b,
                                  uint32_t *bits_out, size_t *launch_sizes, int max_launches)
{
    if (!q || !q->db || q->D == 0 || !bits_a || !bits_out || wave < 0) return VELOPIR_ERR_ARG;
    const int kind = q->kind;
    const bool encdb = kind >= VP_PLAN_INTV_ENCDB && kind <= VP_PLAN_IDM_ENCDB;
    if (kind != VP_QUERY_INTV && kind != VP_QUERY_COV && kind != VP_QUERY_IDM && !encdb) return VELOPIR_ERR_ARG;
    if ((kind == VP_QUERY_INTV || kind == VP_PLAN_INTV_ENCDB) && !bits_b) return VELOPIR_ERR_ARG;
    const int width = q->id_bits;
    if ((kind == VP_QUERY_IDM || kind == VP_PLAN_INTV_ENCDB || kind == VP_PLAN_IDM_ENCDB) && (width < 1 || width > 32))
        return VELOPIR_ERR_ARG;
    if (kind == VP_PLAN_COV_ENCDB && (width < 1 || width > 16)) return VELOPIR_ERR_ARG;
    if (q->payload && (q->payload_bits < 1 || q->payload_bits > 32)) return VELOPIR_ERR_ARG;
    if (q->payload && (kind == VP_QUERY_INTV || kind == VP_QUERY_COV)) return VELOPIR_ERR_ARG;   // no payload form
    if (q->agg_fanin != 0 && (q->agg_fanin < 2 || q->agg_fanin > kMaxFanin || (kind != VP_QUERY_IDM && !encdb)))
        return VELOPIR_ERR_ARG;
    const int fanin = q->agg_fanin >= 2 ? q->agg_fanin : 2;
    if (launch_sizes && max_launches < 0) return VELOPIR_ERR_ARG;

    // stand-in device addresses: distinct, 16-byte aligned, never dereferenced
    uint32_t *in_a = reinterpret_cast<uint32_t *>(uintptr_t(1) << 32);
    uint32_t *in_b = reinterpret_cast<uint32_t *>(uintptr_t(2) << 32);
    uint32_t *out = reinterpret_cast<uint32_t *>(uintptr_t(3) << 32);
    uint32_t *edb = reinterpret_cast<uint32_t *>(uintptr_t(4) << 32);
    uint32_t *epay = reinterpret_cast<uint32_t *>(uintptr_t(5) << 32);
    // query and database widths, in ciphertexts
    const size_t na = kind == VP_QUERY_IDM ? (size_t)width : kind == VP_PLAN_COV_ENCDB ? 2 * (size_t)width
                      : encdb ? (size_t)width : 32;
    const size_t nb = kind == VP_QUERY_INTV ? 32 : kind == VP_PLAN_INTV_ENCDB ? (size_t)width : 0;
    const size_t per_entry = kind == VP_PLAN_INTV_ENCDB ? 4 * (size_t)width : na;   // database ciphertexts per entry
    const int pb = q->payload ? q->payload_bits : 0;
    Program P;
    Builder B(P);
    std::vector<Ref> a(na), b(nb);
    for (size_t i = 0; i < na; ++i) a[i] = B.input(in_a + i * kLweWords);
    for (size_t i = 0; i < nb; ++i) b[i] = B.input(in_b + i * kLweWords);
    switch (kind) {
    case VP_QUERY_INTV: build_intv(B, a.data(), b.data(), q->db, q->D, out); break;
    case VP_QUERY_COV: build_cov(B, a.data(), q->db, q->D, out); break;
    case VP_QUERY_IDM:
        build_idm(B, a.data(), width, q->db, q->D, q->payload, q->payload_bits, out, fanin);
        break;
    case VP_PLAN_INTV_ENCDB:
        build_intv_enc(B, a.data(), b.data(), width, edb, q->D, pb ? epay : nullptr, pb, out, fanin);
        break;
    case VP_PLAN_COV_ENCDB: build_cov_enc(B, a.data(), width, edb, q->D, pb ? epay : nullptr, pb, out, fanin); break;
    default: build_idm_enc(B, a.data(), width, edb, q->D, pb ? epay : nullptr, pb, out, fanin); break;
    }
    relayer(P, wave);
    allocate_slots(P);

    Exec X(P);
    auto enc = [](uint32_t bit) { return bit ? kMu : 0u - kMu; };
    for (size_t i = 0; i < na; ++i) X.write(in_a + i * kLweWords, enc(bits_a[i] & 1u));
    for (size_t i = 0; i < nb; ++i) X.write(in_b + i * kLweWords, enc(bits_b[i] & 1u));
    if (encdb) {   // the database as ServerEnc would encrypt it, one ciphertext per bit, LSB first
        const size_t vals = kind == VP_PLAN_INTV_ENCDB ? 4 : 1, bits = per_entry / vals;
        for (size_t d = 0; d < q->D; ++d)
            for (size_t v = 0; v < vals; ++v)
                for (size_t i = 0; i < bits; ++i)
                    X.write(edb + ((d * vals + v) * bits + i) * kLweWords, enc((q->db[d * vals + v] >> i) & 1u));
        for (size_t d = 0; pb && d < q->D; ++d)
            for (int i = 0; i < pb; ++i)
                X.write(epay + (d * pb + i) * kLweWords, enc((q->payload[d] >> i) & 1u));
    }
    execute(P, X, 0, launch_sizes, max_launches);
    const size_t nout = plan_out_bits(*q);
    for (size_t i = 0; i < nout; ++i) bits_out[i] = (int32_t)X.read(out + i * kLweWords) >= 0 ? 1u : 0u;
    if (X.bad) return VELOPIR_ERR_PLAN;
    return (int)P.layers.size();
}
