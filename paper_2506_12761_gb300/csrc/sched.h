// Gate-layer scheduler: circuits of the three VeLoPIR modes as layered gate
// programs whose every layer is issued as one batch of bootstraps.
//
// A circuit is built over Refs: c = sign * [src] + T(cst), where src is a
// stored ciphertext (device address, or a virtual pool slot) or nothing (a
// trivial ciphertext).  Bootstrap-free gates (NOT, XNOR/AND against a
// plaintext bit, trivial constants) only transform Refs; they are folded into
// the pre-combination of the next bootstrap, which is the same mod-2^32
// arithmetic as materialising them first.  Each bootstrapped gate is placed
// in layer max(ready(inputs)) (as-soon-as-possible), so the layers of many
// database entries and of many queries merge into shared launches.
#pragma once
#include <cstdint>
#include <vector>

#include "vp_internal.h"

namespace vp {

constexpr uint64_t kSlotTag = 1ull << 63;

struct Ref {
    uint64_t src = 0;   // device address, or kSlotTag | virtual slot, or 0 (trivial)
    int32_t sign = 0;
    uint32_t cst = 0;
    int32_t ready = 0;  // the layer index from which src may be read
};

struct Layer {
    std::vector<SumJob> sm;  // multi-input pre-combinations, run before this layer's blind rotations
    std::vector<BrJob> br;   // pointers may carry kSlotTag
    std::vector<KsJob> ks;   // e0/e1 index `br` of this layer
    std::vector<FreeJob> fr; // run after this layer's key switches
};

// The executor splits a layer into chunks whose blind rotations fit its
// extracted-row scratch: gates [g0, g1) of L.ks with rotations [br0, br1).
struct Chunk {
    size_t g0, g1;
    int br0, br1;
};
// Chunks of L for a scratch of `cap` rows (cap <= 0: one chunk).  A gate's
// rotations are never split; a chunk holds at least one gate.
void layer_chunks(const Layer &L, int cap, std::vector<Chunk> &out);
// Chunk size (rotations) of the executor for a program whose largest layer
// has max_br rotations, given a limit of `limit` per launch.  A chunk exceeds
// it only to keep a MUX's two rotations together, so the scratch holds
// max(2, chunk_capacity) rows.
int chunk_capacity(size_t max_br, int limit);

struct Program {
    std::vector<Layer> layers;
    std::vector<FreeJob> pre;   // free gates on inputs, before layer 0
    std::vector<int> slot_def;  // layer whose key switch writes the virtual slot
    std::vector<int> slot_last; // last layer that reads it
    size_t bootstraps = 0;      // blind rotations
    size_t gates = 0;           // key switches
    int nphys = 0;              // physical slots after allocation
    std::vector<int> phys;      // virtual -> physical slot
};

enum GateKind { G_AND = 0, G_NAND, G_OR, G_NOR, G_XOR, G_XNOR, G_ANDNY, G_ANDYN, G_ORNY, G_ORYN, G_MUX };

// Linear pre-combination of a binary gate: T(cst) + s1*c1 + s2*c2.
void gate_combination(int gate, uint32_t *cst, int32_t *s1, int32_t *s2);

class Builder {
public:
    explicit Builder(Program &p) : P(p) {}
    Ref input(const uint32_t *dev) const { Ref r; r.src = (uint64_t)(uintptr_t)dev; r.sign = 1; return r; }
    static Ref trivial(uint32_t mu) { Ref r; r.cst = mu; return r; }
    static Ref neg(const Ref &a) { Ref r = a; r.sign = -a.sign; r.cst = 0u - a.cst; return r; }
    // Bootstrapped binary gate; out == nullptr stores the result in a new pool slot.
    Ref gate(int g, const Ref &a, const Ref &b, uint32_t *out = nullptr);
    // MUX(c, a, b) = c ? a : b with two blind rotations and one key switch.
    Ref mux(const Ref &c, const Ref &a, const Ref &b, uint32_t *out = nullptr);
    // XOR of g >= 2 values with one bootstrap of 2 sum_k in_k + T((g-1)/4)
    // (the fan-in-g HomSum node); more than two stored inputs are summed by a
    // SumJob into a pool slot first.
    Ref xor_many(const Ref *in, int g, uint32_t *out = nullptr);
    // Write the value of a Ref into `out` (device) without a bootstrap.
    void materialize(const Ref &r, uint32_t *out);

private:
    Layer &layer(int i);
    int new_slot(int def);
    void use(const Ref &r, int layer);
    Program &P;
};

// Circuits with a plaintext database (bits LSB first).
// a <= x (plain_first) or x < b, unsigned through the top-bit flip.
Ref build_compare(Builder &B, const Ref *x, int l, uint64_t plain, bool plain_first, bool strict, bool is_unsigned);
Ref build_eq_plain(Builder &B, const Ref *x, int l, uint64_t v, uint32_t *out = nullptr);
void build_intv(Builder &B, const Ref *x, const Ref *y, const uint32_t *rects, size_t D, uint32_t *out);
void build_cov(Builder &B, const Ref *cell, const uint32_t *cells, size_t D, uint32_t *out);
// With a payload, the zeroed payloads are XOR-aggregated by a tree of
// fan-in `fanin` (2: the pairwise HomSum of Section 5; 3..8: one bootstrap
// per fanin inputs).
void build_idm(Builder &B, const Ref *id, int id_bits, const uint32_t *ids, size_t D, const uint32_t *payload,
               int payload_bits, uint32_t *out, int fanin = 2);
constexpr int kMaxFanin = kSumMax;

// Circuits with an encrypted database (the paper's protocol: Alg. ServerEnc
// encrypts every database bit).  Database operands are ciphertexts (device
// pointers, 631 words each, bits LSB first), so the XNORs of the equality
// tests and the XNOR/MUX ripple of the comparators are bootstrapped.
// c1 <= c2 (strict: c1 < c2), l-bit, unsigned through the top-bit flip.
Ref build_compare_enc(Builder &B, const Ref *c1, const Ref *c2, int l, bool strict, bool is_unsigned);
Ref build_eq_enc(Builder &B, const Ref *x, const Ref *y, int l, uint32_t *out = nullptr);
// enc_rects: [D][4][l] ciphertexts (x_lo, x_hi, y_lo, y_hi).  With
// enc_payload ([D][payload_bits] ciphertexts) each entry's payload is zeroed
// by its validation bit and the results are XOR-aggregated into out
// ([payload_bits] ciphertexts) by a tree of fan-in `fanin` (2: Section 5's
// pairwise HomSum); without it out receives the D bits.
void build_intv_enc(Builder &B, const Ref *x, const Ref *y, int l, const uint32_t *enc_rects, size_t D,
                    const uint32_t *enc_payload, int payload_bits, uint32_t *out, int fanin = 2);
// cell: 2w ciphertexts (x then y); enc_cells: [D][2w].
void build_cov_enc(Builder &B, const Ref *cell, int w, const uint32_t *enc_cells, size_t D,
                   const uint32_t *enc_payload, int payload_bits, uint32_t *out, int fanin = 2);
// enc_ids: [D][id_bits].
void build_idm_enc(Builder &B, const Ref *id, int id_bits, const uint32_t *enc_ids, size_t D,
                   const uint32_t *enc_payload, int payload_bits, uint32_t *out, int fanin = 2);

// Wave-filling list schedule (replaces the as-soon-as-possible layers of a
// built program, before allocate_slots).  A gate may run in any launch after
// the launches of the gates it reads; each launch takes, among the ready
// gates, a whole number of full waves (`wave` blind rotations) when at least
// one wave is ready (otherwise everything ready), choosing gates with the
// longest remaining dependency chain first.  The rest waits and merges with
// the gates that become ready.  Results are unchanged (every gate computes
// the same function of the same inputs); wave <= 0 keeps the ASAP layers.
void relayer(Program &p, int wave);

// Liveness-based assignment of virtual slots to physical pool slots: a slot is
// reused only in a layer after the last layer that reads its previous value.
void allocate_slots(Program &p);

}  // namespace vp
