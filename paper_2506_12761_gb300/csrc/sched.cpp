// Gate-layer scheduler for the circuits of VeLoPIR's three modes (see sched.h).
#include "sched.h"

#include <algorithm>
#include <deque>
#include <unordered_map>

namespace vp {

void gate_combination(int gate, uint32_t *cst, int32_t *s1, int32_t *s2)
{
    const uint32_t e = kMu, q = 2 * kMu;  // 1/8, 1/4
    switch (gate) {
    case G_AND:   *cst = 0u - e; *s1 = 1;  *s2 = 1;  break;  // Section 2.2: (0,-1/8)+ct1+ct2
    case G_NAND:  *cst = e;      *s1 = -1; *s2 = -1; break;
    case G_OR:    *cst = e;      *s1 = 1;  *s2 = 1;  break;
    case G_NOR:   *cst = 0u - e; *s1 = -1; *s2 = -1; break;
    case G_XOR:   *cst = q;      *s1 = 2;  *s2 = 2;  break;
    case G_XNOR:  *cst = 0u - q; *s1 = -2; *s2 = -2; break;
    case G_ANDNY: *cst = 0u - e; *s1 = -1; *s2 = 1;  break;
    case G_ANDYN: *cst = 0u - e; *s1 = 1;  *s2 = -1; break;
    case G_ORNY:  *cst = e;      *s1 = -1; *s2 = 1;  break;
    case G_ORYN:  *cst = e;      *s1 = 1;  *s2 = -1; break;
    default:      *cst = 0;      *s1 = 0;  *s2 = 0;  break;
    }
}

Layer &Builder::layer(int i)
{
    while ((int)P.layers.size() <= i) P.layers.emplace_back();
    return P.layers[i];
}

int Builder::new_slot(int def)
{
    P.slot_def.push_back(def);
    P.slot_last.push_back(def);
    return (int)P.slot_def.size() - 1;
}

void Builder::use(const Ref &r, int l)
{
    if (r.src & kSlotTag) {
        const int v = (int)(r.src & ~kSlotTag);
        P.slot_last[v] = std::max(P.slot_last[v], l);
    }
}

static void add_term(BrJob &j, int which, const Ref &r, int32_t g)
{
    const uint32_t *p = reinterpret_cast<const uint32_t *>(r.src);
    const int32_t s = r.src ? g * r.sign : 0;
    if (which == 0) { j.in0 = r.src ? p : nullptr; j.s0 = s; }
    else { j.in1 = r.src ? p : nullptr; j.s1 = s; }
    j.cst += (uint32_t)g * r.cst;
}

Ref Builder::gate(int g, const Ref &a, const Ref &b, uint32_t *out)
{
    const int l = std::max(a.ready, b.ready);
    uint32_t gc;
    int32_t g1, g2;
    gate_combination(g, &gc, &g1, &g2);
    BrJob j{};
    j.cst = gc;
    add_term(j, 0, a, g1);
    add_term(j, 1, b, g2);
    use(a, l);
    use(b, l);
    Layer &L = layer(l);
    KsJob k{};
    k.e0 = (int32_t)L.br.size();
    k.e1 = -1;
    L.br.push_back(j);
    const uint64_t dst = out ? (uint64_t)(uintptr_t)out : (kSlotTag | (uint64_t)new_slot(l));
    k.out = reinterpret_cast<uint32_t *>(dst);
    L.ks.push_back(k);
    P.bootstraps += 1;
    P.gates += 1;
    Ref r;
    r.src = dst;
    r.sign = 1;
    r.ready = l + 1;
    return r;
}

Ref Builder::mux(const Ref &c, const Ref &a, const Ref &b, uint32_t *out)
{
    const int l = std::max(c.ready, std::max(a.ready, b.ready));
    BrJob j0{}, j1{};
    j0.cst = 0u - kMu;                 // AND(c, a)
    add_term(j0, 0, c, 1);
    add_term(j0, 1, a, 1);
    j1.cst = 0u - kMu;                 // AND(NOT c, b)
    add_term(j1, 0, c, -1);
    add_term(j1, 1, b, 1);
    use(c, l);
    use(a, l);
    use(b, l);
    Layer &L = layer(l);
    KsJob k{};
    k.e0 = (int32_t)L.br.size();
    k.e1 = k.e0 + 1;
    k.cst = kMu;                       // + T(1/8) before the key switch
    L.br.push_back(j0);
    L.br.push_back(j1);
    const uint64_t dst = out ? (uint64_t)(uintptr_t)out : (kSlotTag | (uint64_t)new_slot(l));
    k.out = reinterpret_cast<uint32_t *>(dst);
    L.ks.push_back(k);
    P.bootstraps += 2;
    P.gates += 1;
    Ref r;
    r.src = dst;
    r.sign = 1;
    r.ready = l + 1;
    return r;
}

Ref Builder::xor_many(const Ref *in, int g, uint32_t *out)
{
    // One bootstrap of 2 sum_k c_k + T((g-1)/4): phase +1/4 when an odd number
    // of inputs is true, -1/4 when even (g = 2 is the XOR gate's combination).
    int l = 0;
    for (int k = 0; k < g; ++k) l = std::max(l, in[k].ready);
    BrJob j{};
    j.cst = (uint32_t)(g - 1) * (2 * kMu);
    const uint32_t *src[kSumMax];
    int32_t sg[kSumMax];
    int nt = 0;
    for (int k = 0; k < g; ++k) {
        j.cst += 2u * in[k].cst;
        if (in[k].src) {
            src[nt] = reinterpret_cast<const uint32_t *>(in[k].src);
            sg[nt++] = 2 * in[k].sign;
        }
        use(in[k], l);
    }
    if (nt <= 2) {
        if (nt > 0) { j.in0 = src[0]; j.s0 = sg[0]; }
        if (nt > 1) { j.in1 = src[1]; j.s1 = sg[1]; }
    } else {
        const uint64_t t = kSlotTag | (uint64_t)new_slot(l);   // read by this gate's rotation only
        SumJob sj{};
        for (int k = 0; k < nt; ++k) { sj.in[k] = src[k]; sj.s[k] = sg[k]; }
        sj.n = nt;
        sj.out = reinterpret_cast<uint32_t *>(t);
        layer(l).sm.push_back(sj);
        j.in0 = reinterpret_cast<const uint32_t *>(t);
        j.s0 = 1;
    }
    Layer &L = layer(l);
    KsJob k{};
    k.e0 = (int32_t)L.br.size();
    k.e1 = -1;
    L.br.push_back(j);
    const uint64_t dst = out ? (uint64_t)(uintptr_t)out : (kSlotTag | (uint64_t)new_slot(l));
    k.out = reinterpret_cast<uint32_t *>(dst);
    L.ks.push_back(k);
    P.bootstraps += 1;
    P.gates += 1;
    Ref r;
    r.src = dst;
    r.sign = 1;
    r.ready = l + 1;
    return r;
}

void Builder::materialize(const Ref &r, uint32_t *out)
{
    FreeJob f{};
    f.in = r.src ? reinterpret_cast<const uint32_t *>(r.src) : nullptr;
    f.s = r.src ? r.sign : 0;
    f.cst = r.cst;
    f.out = out;
    if (r.ready == 0) {
        P.pre.push_back(f);
    } else {
        use(r, r.ready - 1);
        layer(r.ready - 1).fr.push_back(f);
    }
}

// XNOR against a plaintext bit is free: v ? x : NOT x.
static Ref xnor_plain(const Ref &x, int bit) { return bit ? x : Builder::neg(x); }

Ref build_compare(Builder &B, const Ref *x, int l, uint64_t plain, bool plain_first, bool strict, bool is_unsigned)
{
    // Alg. HomCompLeOPT / HomCompL with the plaintext operand's XNORs and MUXes
    // reduced to one gate each (c ? a : b by cases on the plaintext bit).
    Ref top = x[l - 1];
    if (is_unsigned) {
        plain ^= 1ull << (l - 1);
        top = Builder::neg(top);
    }
    Ref t = Builder::trivial(strict ? 0u - kMu : kMu);
    for (int i = 0; i <= l - 2; ++i) {
        const int bit = (int)((plain >> i) & 1);
        const int g = plain_first ? (bit ? G_AND : G_OR) : (bit ? G_ORNY : G_ANDNY);
        t = B.gate(g, x[i], t);
    }
    const int tb = (int)((plain >> (l - 1)) & 1);
    const int g = plain_first ? (tb ? G_ORNY : G_ANDNY) : (tb ? G_AND : G_OR);
    return B.gate(g, top, t);
}

Ref build_eq_plain(Builder &B, const Ref *x, int l, uint64_t v, uint32_t *out)
{
    // Alg. HomEqOPT: free XNORs, then t[i] = AND(t[i], t[i+k]) for k = 1, 2, 4, ...
    std::vector<Ref> t(l);
    for (int i = 0; i < l; ++i) t[i] = xnor_plain(x[i], (int)((v >> i) & 1));
    int last_k = 0;
    for (int k = 1; k < l; k *= 2) last_k = k;
    for (int k = 1; k < l; k *= 2)
        for (int i = 0; i + k < l; i += 2 * k)
            t[i] = B.gate(G_AND, t[i], t[i + k], (out && k == last_k && i == 0) ? out : nullptr);
    if (out && l == 1) B.materialize(t[0], out);
    return t[0];
}

void build_intv(Builder &B, const Ref *x, const Ref *y, const uint32_t *rects, size_t D, uint32_t *out)
{
    // Alg. InterValid: v = AND(AND(LE(x_lo,x), L(x,x_hi)), AND(LE(y_lo,y), L(y,y_hi))).
    for (size_t d = 0; d < D; ++d) {
        const uint32_t *r = rects + 4 * d;
        Ref vxl = build_compare(B, x, 32, r[0], true, false, true);
        Ref vxr = build_compare(B, x, 32, r[1], false, true, true);
        Ref vyl = build_compare(B, y, 32, r[2], true, false, true);
        Ref vyr = build_compare(B, y, 32, r[3], false, true, true);
        Ref vx = B.gate(G_AND, vxl, vxr);
        Ref vy = B.gate(G_AND, vyl, vyr);
        B.gate(G_AND, vx, vy, out + d * kLweWords);
    }
}

void build_cov(Builder &B, const Ref *cell, const uint32_t *cells, size_t D, uint32_t *out)
{
    // Alg. CoV: AND(HomEqOPT(x, loc_x), HomEqOPT(y, loc_y)), 16 + 16 bits.
    for (size_t d = 0; d < D; ++d) {
        Ref vx = build_eq_plain(B, cell, 16, cells[d] & 0xFFFFu);
        Ref vy = build_eq_plain(B, cell + 16, 16, cells[d] >> 16);
        B.gate(G_AND, vx, vy, out + d * kLweWords);
    }
}

// XOR over the D entries of S[d * bits + j], per bit j, into out[j]: Section
// 5's pairwise HomSum tree (fanin 2), or the fan-in-g tree whose nodes XOR g
// values with one bootstrap (Builder::xor_many).  D = 1 writes nothing.
static void xor_tree(Builder &B, std::vector<Ref> &S, size_t D, int bits, uint32_t *out, int fanin)
{
    if (fanin > 2) {
        // for k = 1, g, g^2, ... the members i, i + k, ..., i + (g-1)k (those
        // below D) of each group are XORed into member i; the level with
        // g k >= D writes `out`
        const size_t g = (size_t)std::min(fanin, kMaxFanin);
        Ref grp[kMaxFanin];
        for (size_t k = 1; k < D; k *= g)
            for (size_t i = 0; i < D; i += g * k) {
                size_t m = 0;
                while (m < g && i + m * k < D) ++m;
                if (m < 2) continue;
                for (int j = 0; j < bits; ++j) {
                    for (size_t q = 0; q < m; ++q) grp[q] = S[(i + q * k) * bits + j];
                    uint32_t *o = (g * k >= D && i == 0) ? out + (size_t)j * kLweWords : nullptr;
                    S[i * bits + j] = B.xor_many(grp, (int)m, o);
                }
            }
        return;
    }
    size_t last_k = 0;
    for (size_t k = 1; k < D; k *= 2) last_k = k;
    for (size_t k = 1; k < D; k *= 2)
        for (size_t i = 0; i + k < D; i += 2 * k)
            for (int j = 0; j < bits; ++j) {
                uint32_t *o = (k == last_k && i == 0) ? out + (size_t)j * kLweWords : nullptr;
                S[i * bits + j] = B.gate(G_XOR, S[i * bits + j], S[(i + k) * bits + j], o);
            }
}

void build_idm(Builder &B, const Ref *id, int id_bits, const uint32_t *ids, size_t D, const uint32_t *payload,
               int payload_bits, uint32_t *out, int fanin)
{
    if (!payload) {
        for (size_t d = 0; d < D; ++d) build_eq_plain(B, id, id_bits, ids[d], out + d * kLweWords);
        return;
    }
    // Match bits, free zero-out with each plaintext payload bit (Alg.
    // HomBitwiseAND: AND(v, 1) = v, AND(v, 0) = Enc(0) trivially), then the
    // pairwise HomSum XOR reduction of Section 5 per payload bit.
    std::vector<Ref> v(D);
    for (size_t d = 0; d < D; ++d) v[d] = build_eq_plain(B, id, id_bits, ids[d]);
    std::vector<Ref> S(D * (size_t)payload_bits);
    for (size_t d = 0; d < D; ++d)
        for (int j = 0; j < payload_bits; ++j)
            S[d * payload_bits + j] = ((payload[d] >> j) & 1u) ? v[d] : Builder::trivial(0u - kMu);
    xor_tree(B, S, D, payload_bits, out, fanin);
    if (D == 1)
        for (int j = 0; j < payload_bits; ++j) B.materialize(S[j], out + (size_t)j * kLweWords);
}

Ref build_compare_enc(Builder &B, const Ref *c1, const Ref *c2, int l, bool strict, bool is_unsigned)
{
    // Alg. HomCompLeOPT (HomCompL for strict) with both operands encrypted:
    // t0 = XOR of the top bits; t1 = T(+-1/8); t1 = MUX(XNOR(c1_i, c2_i), t1, c2_i)
    // for i = 0..l-2 (the XNORs are independent, the MUXes ripple); the result
    // is MUX(t0, c1_top, t1).  Signed two's complement as in the paper; the
    // unsigned form flips both top bits first (free NOTs).
    Ref top1 = c1[l - 1], top2 = c2[l - 1];
    if (is_unsigned) {
        top1 = Builder::neg(top1);
        top2 = Builder::neg(top2);
    }
    const Ref t0 = B.gate(G_XOR, top1, top2);
    std::vector<Ref> tx(l > 1 ? l - 1 : 0);
    for (int i = 0; i + 1 < l; ++i) tx[i] = B.gate(G_XNOR, c1[i], c2[i]);
    Ref t1 = Builder::trivial(strict ? 0u - kMu : kMu);
    for (int i = 0; i + 1 < l; ++i) t1 = B.mux(tx[i], t1, c2[i]);
    return B.mux(t0, top1, t1);
}

Ref build_eq_enc(Builder &B, const Ref *x, const Ref *y, int l, uint32_t *out)
{
    // Alg. HomEqOPT with both operands encrypted: bootstrapped XNORs, then the
    // pairwise AND reduction t[i] = AND(t[i], t[i+k]) for k = 1, 2, 4, ...
    std::vector<Ref> t(l);
    for (int i = 0; i < l; ++i) t[i] = B.gate(G_XNOR, x[i], y[i], (out && l == 1) ? out : nullptr);
    int last_k = 0;
    for (int k = 1; k < l; k *= 2) last_k = k;
    for (int k = 1; k < l; k *= 2)
        for (int i = 0; i + k < l; i += 2 * k)
            t[i] = B.gate(G_AND, t[i], t[i + k], (out && k == last_k && i == 0) ? out : nullptr);
    return t[0];
}

static std::vector<Ref> enc_inputs(Builder &B, const uint32_t *base, int count)
{
    std::vector<Ref> r(count);
    for (int i = 0; i < count; ++i) r[i] = B.input(base + (size_t)i * kLweWords);
    return r;
}

// Alg. HomBitwiseAND with encrypted payloads (one bootstrapped AND of the
// validation bit with each payload bit), then the pairwise HomSum XOR
// reduction of Section 5 per payload bit into out.
static void aggregate_enc(Builder &B, const std::vector<Ref> &v, const uint32_t *enc_payload, int payload_bits,
                          uint32_t *out, int fanin)
{
    const size_t D = v.size();
    std::vector<Ref> S(D * (size_t)payload_bits);
    for (size_t d = 0; d < D; ++d) {
        const std::vector<Ref> pay = enc_inputs(B, enc_payload + d * (size_t)payload_bits * kLweWords, payload_bits);
        for (int j = 0; j < payload_bits; ++j)
            S[d * payload_bits + j] = B.gate(G_AND, v[d], pay[j], (D == 1) ? out + (size_t)j * kLweWords : nullptr);
    }
    xor_tree(B, S, D, payload_bits, out, fanin);
}

void build_intv_enc(Builder &B, const Ref *x, const Ref *y, int l, const uint32_t *enc_rects, size_t D,
                    const uint32_t *enc_payload, int payload_bits, uint32_t *out, int fanin)
{
    // Alg. InterValid with encrypted bounds: AND(AND(LE(x_lo,x), L(x,x_hi)), AND(LE(y_lo,y), L(y,y_hi))).
    std::vector<Ref> v(D);
    for (size_t d = 0; d < D; ++d) {
        const std::vector<Ref> r = enc_inputs(B, enc_rects + d * 4 * (size_t)l * kLweWords, 4 * l);
        Ref vxl = build_compare_enc(B, r.data(), x, l, false, true);
        Ref vxr = build_compare_enc(B, x, r.data() + l, l, true, true);
        Ref vyl = build_compare_enc(B, r.data() + 2 * l, y, l, false, true);
        Ref vyr = build_compare_enc(B, y, r.data() + 3 * l, l, true, true);
        Ref vx = B.gate(G_AND, vxl, vxr);
        Ref vy = B.gate(G_AND, vyl, vyr);
        v[d] = B.gate(G_AND, vx, vy, enc_payload ? nullptr : out + d * kLweWords);
    }
    if (enc_payload) aggregate_enc(B, v, enc_payload, payload_bits, out, fanin);
}

void build_cov_enc(Builder &B, const Ref *cell, int w, const uint32_t *enc_cells, size_t D,
                   const uint32_t *enc_payload, int payload_bits, uint32_t *out, int fanin)
{
    // Alg. CoV with encrypted cells: AND(HomEqOPT(x, loc_x), HomEqOPT(y, loc_y)).
    std::vector<Ref> v(D);
    for (size_t d = 0; d < D; ++d) {
        const std::vector<Ref> c = enc_inputs(B, enc_cells + d * 2 * (size_t)w * kLweWords, 2 * w);
        Ref vx = build_eq_enc(B, cell, c.data(), w);
        Ref vy = build_eq_enc(B, cell + w, c.data() + w, w);
        v[d] = B.gate(G_AND, vx, vy, enc_payload ? nullptr : out + d * kLweWords);
    }
    if (enc_payload) aggregate_enc(B, v, enc_payload, payload_bits, out, fanin);
}

void build_idm_enc(Builder &B, const Ref *id, int id_bits, const uint32_t *enc_ids, size_t D,
                   const uint32_t *enc_payload, int payload_bits, uint32_t *out, int fanin)
{
    std::vector<Ref> v(D);
    for (size_t d = 0; d < D; ++d) {
        const std::vector<Ref> c = enc_inputs(B, enc_ids + d * (size_t)id_bits * kLweWords, id_bits);
        v[d] = build_eq_enc(B, id, c.data(), id_bits, enc_payload ? nullptr : out + d * kLweWords);
    }
    if (enc_payload) aggregate_enc(B, v, enc_payload, payload_bits, out, fanin);
}

void layer_chunks(const Layer &L, int cap, std::vector<Chunk> &out)
{
    out.clear();
    const size_t nks = L.ks.size();
    size_t g = 0;
    while (g < nks) {
        const int br0 = L.ks[g].e0;
        size_t g1 = g;
        int br1 = br0;
        while (g1 < nks) {
            const int hi = std::max(L.ks[g1].e0, L.ks[g1].e1) + 1;
            if (cap > 0 && hi - br0 > cap && g1 > g) break;
            br1 = std::max(br1, hi);
            ++g1;
        }
        out.push_back({g, g1, br0, br1});
        g = g1;
    }
}

int chunk_capacity(size_t max_br, int limit)
{
    // a chunk always holds a whole gate, so a MUX's two rotations need two
    // rows of scratch even under a limit of one
    return (int)std::min<size_t>(std::max<size_t>(1, max_br), (size_t)std::max(1, limit));
}

void relayer(Program &p, int wave)
{
    if (wave <= 0 || p.layers.size() <= 1) return;
    struct G {
        int layer, ks, nbr, height = 1, indeg = 0, at = -1;
    };
    std::vector<G> g;
    // Producer of each readable value: pool slots are dense indices (a flat
    // table); device addresses (outputs into caller buffers) are few (a map).
    std::vector<int> slot_prod(p.slot_def.size(), -1);
    std::unordered_map<uint64_t, int> addr_prod;
    auto set_prod = [&](const void *a, int gate) {
        const uint64_t v = (uint64_t)(uintptr_t)a;
        if (v & kSlotTag) slot_prod[v & ~kSlotTag] = gate;
        else addr_prod[v] = gate;
    };
    auto prod_of = [&](const void *a) -> int {
        const uint64_t v = (uint64_t)(uintptr_t)a;
        if (!v) return -1;
        if (v & kSlotTag) return slot_prod[v & ~kSlotTag];
        auto it = addr_prod.find(v);
        return it == addr_prod.end() ? -1 : it->second;
    };
    for (int l = 0; l < (int)p.layers.size(); ++l) {
        const Layer &L = p.layers[l];
        for (int k = 0; k < (int)L.ks.size(); ++k) {
            G x;
            x.layer = l;
            x.ks = k;
            x.nbr = L.ks[k].e1 >= 0 ? 2 : 1;
            set_prod(L.ks[k].out, (int)g.size());
            g.push_back(x);
        }
        // a free job's output is ready with its input's producer
        for (const FreeJob &f : L.fr) {
            const int q = prod_of(f.in);
            if (q >= 0) set_prod(f.out, q);
        }
    }
    const int ng = (int)g.size();
    // The multi-input pre-combination feeding a rotation, by its pool slot.
    std::unordered_map<uint64_t, const SumJob *> sum_of;
    for (const Layer &L : p.layers)
        for (const SumJob &sj : L.sm) sum_of[(uint64_t)(uintptr_t)sj.out] = &sj;
    auto sum_for = [&](const uint32_t *in) -> const SumJob * {
        if (sum_of.empty() || !in) return nullptr;
        auto it = sum_of.find((uint64_t)(uintptr_t)in);
        return it == sum_of.end() ? nullptr : it->second;
    };
    // predecessors (at most 2 rotations x 2 inputs, or the kSumMax inputs of
    // a pre-combination), then successors in CSR form
    constexpr int kMaxPred = 2 * kSumMax;
    std::vector<int> pred(kMaxPred * (size_t)ng, -1);
    std::vector<int> nsucc(ng + 1, 0);
    for (int i = 0; i < ng; ++i) {
        const Layer &L = p.layers[g[i].layer];
        const KsJob &k = L.ks[g[i].ks];
        int np = 0;
        auto add = [&](const uint32_t *in) {
            const int q = prod_of(in);
            if (q < 0 || q == i) return;
            bool dup = false;
            for (int t = 0; t < np; ++t) dup |= pred[kMaxPred * (size_t)i + t] == q;
            if (!dup && np < kMaxPred) pred[kMaxPred * (size_t)i + np++] = q;
        };
        for (int e : {k.e0, k.e1}) {
            if (e < 0) continue;
            for (const uint32_t *in : {L.br[e].in0, L.br[e].in1}) {
                if (const SumJob *sj = sum_for(in)) {
                    for (int t = 0; t < sj->n; ++t) add(sj->in[t]);
                } else {
                    add(in);
                }
            }
        }
        g[i].indeg = np;
        for (int t = 0; t < np; ++t) nsucc[pred[kMaxPred * (size_t)i + t] + 1]++;
    }
    for (int i = 0; i < ng; ++i) nsucc[i + 1] += nsucc[i];
    std::vector<int> succ(nsucc[ng]);
    {
        std::vector<int> fill(nsucc.begin(), nsucc.end() - 1);
        for (int i = 0; i < ng; ++i)
            for (int t = 0; t < kMaxPred && pred[kMaxPred * (size_t)i + t] >= 0; ++t)
                succ[fill[pred[kMaxPred * (size_t)i + t]]++] = i;
    }
    // longest chain of gates from each gate to the end (producers precede
    // consumers in the ASAP order, so a reverse sweep sees successors first)
    int hmax = 1;
    for (int i = ng - 1; i >= 0; --i) {
        for (int e = nsucc[i]; e < nsucc[i + 1]; ++e) g[i].height = std::max(g[i].height, 1 + g[succ[e]].height);
        hmax = std::max(hmax, g[i].height);
    }
    std::vector<std::deque<int>> ready(hmax + 1);
    size_t nready = 0;
    for (int i = 0; i < ng; ++i)
        if (g[i].indeg == 0) { ready[g[i].height].push_back(i); nready += g[i].nbr; }
    std::vector<std::vector<int>> sched;
    std::vector<int> next;
    int done = 0;
    while (done < ng) {
        const size_t cap = nready >= (size_t)wave ? nready / wave * wave : nready;
        std::vector<int> take;
        size_t used = 0;
        for (int h = hmax; h >= 1 && used < cap; --h) {
            auto &q = ready[h];
            while (!q.empty() && used + g[q.front()].nbr <= cap) {
                take.push_back(q.front());
                used += g[q.front()].nbr;
                q.pop_front();
            }
        }
        if (take.empty())   // only a two-rotation gate is ready and cap is odd: take it anyway
            for (int h = hmax; h >= 1 && take.empty(); --h)
                if (!ready[h].empty()) { take.push_back(ready[h].front()); used += g[take[0]].nbr; ready[h].pop_front(); }
        nready -= used;
        const int t = (int)sched.size();
        next.clear();
        for (int i : take) {
            g[i].at = t;
            for (int e = nsucc[i]; e < nsucc[i + 1]; ++e)
                if (--g[succ[e]].indeg == 0) next.push_back(succ[e]);
        }
        for (int s : next) { ready[g[s].height].push_back(s); nready += g[s].nbr; }
        done += (int)take.size();
        sched.push_back(std::move(take));
    }

    // rebuild the layers, the free jobs after their producer's layer, and slot liveness
    // free jobs of each producer gate (usually none): a sorted list
    std::vector<std::pair<int, FreeJob>> fr_of;
    for (const Layer &L : p.layers)
        for (const FreeJob &f : L.fr) {
            const int q = prod_of(f.in);
            if (q >= 0) fr_of.emplace_back(q, f);
            else p.pre.push_back(f);
        }
    std::stable_sort(fr_of.begin(), fr_of.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
    std::vector<Layer> NL(sched.size());
    for (size_t t = 0; t < sched.size(); ++t) {
        size_t nbr = 0;
        for (int i : sched[t]) nbr += g[i].nbr;
        NL[t].br.reserve(nbr);
        NL[t].ks.reserve(sched[t].size());
    }
    for (size_t t = 0; t < sched.size(); ++t)
        for (int i : sched[t]) {
            const Layer &L = p.layers[g[i].layer];
            KsJob k = L.ks[g[i].ks];
            const int e0 = (int)NL[t].br.size();
            NL[t].br.push_back(L.br[k.e0]);
            if (k.e1 >= 0) NL[t].br.push_back(L.br[k.e1]);
            for (int e : {k.e0, k.e1})   // a rotation's pre-combination runs in its launch
                if (e >= 0)
                    for (const uint32_t *in : {L.br[e].in0, L.br[e].in1})
                        if (const SumJob *sj = sum_for(in)) NL[t].sm.push_back(*sj);
            k.e0 = e0;
            k.e1 = k.e1 >= 0 ? e0 + 1 : -1;
            NL[t].ks.push_back(k);
            auto it = std::lower_bound(fr_of.begin(), fr_of.end(), i,
                                       [](const std::pair<int, FreeJob> &a, int v) { return a.first < v; });
            for (; it != fr_of.end() && it->first == i; ++it) NL[t].fr.push_back(it->second);
        }
    p.layers.swap(NL);
    auto slot_of = [](const void *a) { return ((uint64_t)(uintptr_t)a & kSlotTag) ? (int)((uint64_t)(uintptr_t)a & ~kSlotTag) : -1; };
    for (int l = 0; l < (int)p.layers.size(); ++l) {
        const Layer &L = p.layers[l];
        for (const KsJob &k : L.ks)
            if (int v = slot_of(k.out); v >= 0) p.slot_def[v] = p.slot_last[v] = l;
        for (const SumJob &sj : L.sm)
            if (int v = slot_of(sj.out); v >= 0) p.slot_def[v] = p.slot_last[v] = l;
    }
    for (int l = 0; l < (int)p.layers.size(); ++l) {
        const Layer &L = p.layers[l];
        for (const SumJob &sj : L.sm)
            for (int t = 0; t < sj.n; ++t)
                if (int v = slot_of(sj.in[t]); v >= 0) p.slot_last[v] = std::max(p.slot_last[v], l);
        for (const BrJob &j : L.br)
            for (const uint32_t *in : {j.in0, j.in1})
                if (int v = in ? slot_of(in) : -1; v >= 0) p.slot_last[v] = std::max(p.slot_last[v], l);
        for (const FreeJob &f : L.fr)
            if (int v = f.in ? slot_of(f.in) : -1; v >= 0) p.slot_last[v] = std::max(p.slot_last[v], l);
    }
}

void allocate_slots(Program &p)
{
    const int nv = (int)p.slot_def.size();
    const int nl = (int)p.layers.size();
    std::vector<std::vector<int>> defs(nl + 1), lasts(nl + 1);
    for (int v = 0; v < nv; ++v) {
        defs[p.slot_def[v]].push_back(v);
        lasts[p.slot_last[v]].push_back(v);
    }
    p.phys.assign(nv, -1);
    std::vector<int> freelist;
    int next = 0;
    for (int l = 0; l < nl; ++l) {
        if (l > 0)
            for (int v : lasts[l - 1]) freelist.push_back(p.phys[v]);
        for (int v : defs[l]) {
            if (!freelist.empty()) { p.phys[v] = freelist.back(); freelist.pop_back(); }
            else p.phys[v] = next++;
        }
    }
    p.nphys = next;
}

}  // namespace vp
