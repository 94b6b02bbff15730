"""The C-ABI library loads, exports every symbol include/velopir.h declares,
and its host-only client functions agree bit for bit with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from conftest import ROOT
from paper_2506_12761_gb300 import build, synth
from paper_2506_12761_gb300 import velopir as vp


@pytest.fixture(scope="module")
def lib():
    build.build()
    return vp.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "velopir.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(velopir_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    decl = declared_symbols()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(vp.EXPORTS) == decl


def test_create_without_gpu_fails_cleanly(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is visible")
    except ImportError:
        pass
    h = ctypes.c_void_p(1)
    rc = lib.velopir_create(ctypes.byref(h), 0, 0, None)
    assert rc in (-7, -4) and h.value is None
    assert lib.velopir_last_error(None)


def test_null_context_is_an_argument_error(lib):
    assert lib.velopir_bootstrap_batch(None, 0, None, None, 1) == -1
    assert lib.velopir_sync(None) == -1
    assert lib.velopir_destroy(None) == 0


def test_client_keygen_matches_oracle(lib, paper_keys):
    km = synth.key_material()
    bk, ksk = vp.velopir_client_keygen(km)
    assert np.array_equal(bk, paper_keys.bk.reshape(-1))
    assert np.array_equal(ksk, paper_keys.ksk.reshape(-1))


def test_client_encrypt_decrypt_matches_oracle(lib, paper_keys):
    bits = synth.Stream(9, 2, 1).bits(100)
    lm = synth.lwe_material(100, seed=9)
    ct = vp.velopir_client_encrypt_bits(paper_keys.s, bits, lm)
    assert np.array_equal(ct, oracle.encrypt_bits(paper_keys.s, bits, lm))
    assert np.array_equal(vp.velopir_client_decrypt_bits(paper_keys.s, ct), bits)
    assert np.array_equal(vp.velopir_client_decrypt_bits(paper_keys.s, ct), oracle.decrypt_bits(paper_keys.s, ct))


def test_client_rejects_other_parameters(lib):
    p = vp.Params(500, 1024, 1, 3, 7, 8, 2)
    z = np.zeros(16, dtype=np.uint32)
    assert lib.velopir_client_keygen(ctypes.byref(p), *(vp.ptr(z),) * 8) == -1
