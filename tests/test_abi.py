"""The two C-ABI libraries load and export every symbol their headers
declare: libvelopir.so (include/velopir.h, the GPU library) and
libvelopir_client.so (include/velopir_client.h, host only: it links no CUDA
library); the client functions agree bit for bit with the oracle."""
import ctypes
import os
import re
import shutil
import subprocess

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


@pytest.fixture(scope="module")
def clib():
    build.build()
    return vp.clib()


def declared_symbols(header="velopir.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(velopir_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    decl = declared_symbols()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(vp.EXPORTS) == decl


def test_client_library_exports_its_header_and_the_gpu_library_does_not(lib, clib):
    decl = declared_symbols("velopir_client.h")
    assert sorted(vp.CLIENT_EXPORTS) == decl and len(decl) == 5
    for name in decl:
        assert hasattr(clib, name), name
    gpu = ctypes.CDLL(build.LIB)
    for name in decl:
        assert not hasattr(gpu, name), f"{name} is exported by the GPU library"
    assert not set(decl) & set(declared_symbols())


def test_client_library_needs_no_cuda(clib):
    """Its dynamic dependencies name no CUDA library, and a fresh interpreter
    that loads it and encrypts and decrypts has no CUDA library mapped."""
    if shutil.which("ldd"):
        deps = subprocess.run(["ldd", build.CLIENT_LIB], capture_output=True, text=True).stdout
        assert "cuda" not in deps.lower(), deps
    code = ("import ctypes, numpy as np; L = ctypes.CDLL(%r); "
            "s = np.zeros(630, np.uint32); a = np.zeros(630, np.uint32); e = np.zeros(1, np.uint32); "
            "b = np.ones(1, np.uint32); ct = np.zeros(631, np.uint32); o = np.zeros(1, np.uint32); "
            "p = lambda x: x.ctypes.data_as(ctypes.c_void_p); "
            "assert L.velopir_client_encrypt_bits(p(s), p(b), p(a), p(e), ctypes.c_size_t(1), p(ct)) == 0; "
            "assert L.velopir_client_decrypt_bits(p(s), p(ct), ctypes.c_size_t(1), p(o)) == 0 and o[0] == 1; "
            "maps = open('/proc/self/maps').read(); assert 'libcuda' not in maps, 'CUDA mapped'; print('ok')"
            ) % build.CLIENT_LIB
    r = subprocess.run(["python3", "-c", code], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr


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
    # the client preprocessing on the GPU checks its context before any CUDA call
    p = vp.paper_params()
    assert lib.velopir_gpu_keygen(None, ctypes.byref(p), None, None, None, None, None, None, None, None) == -1
    assert lib.velopir_gpu_encrypt_bits(None, None, None, None, None, 1, None) == -1
    assert lib.velopir_gpu_pubkeygen(None, None, None, None, 1, None) == -1
    assert lib.velopir_gpu_server_encrypt(None, None, None, 1, None) == -1


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


def test_client_rejects_other_parameters(clib):
    p = vp.Params(500, 1024, 1, 3, 7, 8, 2)
    z = np.zeros(16, dtype=np.uint32)
    assert clib.velopir_client_keygen(ctypes.byref(p), *(vp.ptr(z),) * 8) == -1
