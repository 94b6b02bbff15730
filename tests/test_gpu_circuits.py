"""GPU parity of the three mode circuits against the oracle, bit for bit,
through the C ABI; plus decryption against the plaintext predicates."""
import numpy as np
import pytest

import oracle
from gpu_common import encrypt_value_bits, gpu_ctx, make_queries, oracle_out
from paper_2506_12761_gb300 import synth
from paper_2506_12761_gb300 import velopir as vp

pytestmark = pytest.mark.gpu


def test_idm8_d4_whole_circuit(paper_keys):
    """Identifier matching, 8-bit id, D = 4 (28 bootstraps in layers 16/8/4)."""
    ctx, s = gpu_ctx()
    w = synth.idm_workload(4, 8)
    x = encrypt_value_bits(s, w["query"], 8, 500)
    ids = w["ids"].astype(np.uint32)
    out = np.zeros((4, 631), dtype=np.uint32)
    vp.velopir_id_match(ctx.h, x, 8, ids, 4, None, 0, out)
    assert np.array_equal(out, oracle.idm_batch(paper_keys, x, ids))
    assert list(vp.velopir_client_decrypt_bits(s, out)) == [int(i == w["query"]) for i in ids]


def _intv_small(paper_keys, s):
    """The serving tests' two-rectangle IntV query (the first rectangle
    contains the point) and the oracle's whole circuit on it, from the shared
    oracle runs."""
    q = make_queries(s, 3)[0]
    return dict(w=q["w"], rects=q["db"], cx=q["a"], cy=q["b"], D=q["D"], want=oracle_out(paper_keys, q))


def test_intv_small_whole_circuit(paper_keys):
    ctx, s = gpu_ctx()
    c = _intv_small(paper_keys, s)
    w, rects = c["w"], c["rects"]
    out = np.zeros((c["D"], 631), dtype=np.uint32)
    vp.velopir_interval_query(ctx.h, c["cx"], c["cy"], rects, c["D"], out)
    assert np.array_equal(out, c["want"])
    want = [int(r[0] <= w["x"] < r[1] and r[2] <= w["y"] < r[3]) for r in rects.astype(np.int64)]
    assert list(vp.velopir_client_decrypt_bits(s, out)) == want and want[0] == 1


def test_cov_small_whole_circuit(paper_keys):
    ctx, s = gpu_ctx()
    w = synth.cov_workload(3, substream=2)
    cell = encrypt_value_bits(s, w["cell"], 32, 503)
    cells = w["cells"].astype(np.uint32)
    out = np.zeros((3, 631), dtype=np.uint32)
    vp.velopir_coordinate_query(ctx.h, cell, cells, 3, out)
    assert np.array_equal(out, oracle.cov_batch(paper_keys, cell, cells))
    assert list(vp.velopir_client_decrypt_bits(s, out)) == [int(c == w["cell"]) for c in cells]


def test_idm32_payload_aggregation(paper_keys):
    ctx, s = gpu_ctx()
    w = synth.idm_workload(5, 32, distinct=True, payload=True, substream=3)
    x = encrypt_value_bits(s, w["query"], 32, 504)
    ids = w["ids"].astype(np.uint32)
    pay = w["payload"].astype(np.uint32)
    out = np.zeros((32, 631), dtype=np.uint32)
    vp.velopir_id_match(ctx.h, x, 32, ids, 5, pay, 32, out)
    assert np.array_equal(out, oracle.idm_payload(paper_keys, x, ids, pay, 32))
    got = vp.velopir_client_decrypt_bits(s, out)
    assert int(sum(int(b) << j for j, b in enumerate(got))) == int(pay[w["planted"]])


def test_degenerate_shapes(paper_keys):
    ctx, s = gpu_ctx()
    # id_bits = 1: no bootstrap at all (plaintext XNOR is free)
    x = encrypt_value_bits(s, 1, 1, 505)
    out = np.zeros((2, 631), dtype=np.uint32)
    vp.velopir_id_match(ctx.h, x, 1, np.array([1, 0], dtype=np.uint32), 2, None, 0, out)
    assert np.array_equal(out, oracle.idm_batch(paper_keys, x, [1, 0]))
    # D = 1 with payload: no XOR layer
    x = encrypt_value_bits(s, 3, 2, 506)
    out = np.zeros((4, 631), dtype=np.uint32)
    vp.velopir_id_match(ctx.h, x, 2, np.array([3], dtype=np.uint32), 1, np.array([9], dtype=np.uint32), 4, out)
    assert np.array_equal(out, oracle.idm_payload(paper_keys, x, [3], [9], 4))
    # D = 0: nothing to do
    vp.velopir_id_match(ctx.h, x, 2, np.zeros(1, dtype=np.uint32), 0, None, 0, out)


def test_device_resident_database(paper_keys):
    """Ciphertexts, database and output all in device memory (the workload of
    test_intv_small_whole_circuit, checked against the same oracle run)."""
    import torch
    ctx, s = gpu_ctx()
    c = _intv_small(paper_keys, s)
    dx, dy = (torch.from_numpy(a.view(np.int32)).cuda() for a in (c["cx"], c["cy"]))
    dr = torch.from_numpy(c["rects"].view(np.int32)).cuda()
    dout = torch.zeros((c["D"], 631), dtype=torch.int32, device="cuda")
    vp.velopir_interval_query(ctx.h, dx, dy, dr, c["D"], dout)
    out = dout.cpu().numpy().view(np.uint32)
    assert np.array_equal(out, c["want"])


def test_launch_limit_one_is_one_bootstrap_per_launch(paper_keys):
    """velopir_set_launch_limit(1): every blind-rotation launch holds one
    gate (the plain baseline of a whole query); the ciphertexts equal the
    layer-batched ones and the oracle's."""
    ctx, s = gpu_ctx()
    w = synth.idm_workload(4, 8)
    x = encrypt_value_bits(s, w["query"], 8, 507)
    ids = w["ids"].astype(np.uint32)
    batched = np.zeros((4, 631), dtype=np.uint32)
    vp.velopir_id_match(ctx.h, x, 8, ids, 4, None, 0, batched)
    plain = np.zeros_like(batched)
    vp.velopir_set_launch_limit(ctx.h, 1)
    try:
        vp.velopir_profile(ctx.h, True)
        vp.velopir_id_match(ctx.h, x, 8, ids, 4, None, 0, plain)
        launches, rotations, _ = vp.velopir_profile_read(ctx.h, vp.VP_KERNEL_BLIND_ROTATE)
        vp.velopir_profile(ctx.h, False)
    finally:
        vp.velopir_set_launch_limit(ctx.h, 0)
    assert rotations == 28 and launches == 28
    assert np.array_equal(plain, batched)
    assert np.array_equal(plain, oracle.idm_batch(paper_keys, x, ids))
