"""The C-ABI library builds, loads and exports every symbol include/bbc.h
declares; host-side argument checks answer before any device work.

No test here calls into the GPU."""

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2604_01960_gb300 as bbc
    bbc.build()
    return bbc.lib()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "bbc.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(bbc_\w+)\s*\(", txt, flags=re.M)))


def test_header_and_binding_agree():
    import paper_2604_01960_gb300 as bbc
    assert declared_symbols() == sorted(bbc.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert lib.bbc_version().decode().startswith("bbc-gb300")


def test_null_and_bad_arguments_rejected_without_device(lib):
    import paper_2604_01960_gb300 as bbc
    assert lib.bbc_index_create(None, 0, None) == -1
    assert lib.bbc_search(None, None, 1, 10, 4, None, None, None) == -1
    assert lib.bbc_set_param(None, b"kc_ratio", 2.0) == -1
    assert lib.bbc_index_free(None) == -1
    assert lib.bbc_index_load(None, 0, None) == -1
    assert lib.bbc_index_load(b"/nonexistent/index.bin", 0, C.byref(C.c_void_p())) == -2
    assert "cannot open" in lib.bbc_last_error().decode()
    with pytest.raises(bbc.BBCError):
        bbc._check(-9)


def _host(n=64, d=16, L=4, M=8, bits=8):
    rng = np.random.default_rng(0)
    offs = np.linspace(0, n, L + 1).astype(np.int64)
    return dict(n=n, d=d, L=L, M=M, bits=bits,
                cent=rng.standard_normal((L, d)).astype(np.float32), offs=offs,
                ids=np.arange(n, dtype=np.int64), codes=rng.integers(0, 256, (n, M * bits // 8)).astype(np.uint8),
                books=rng.standard_normal((M, 1 << bits, d // M)).astype(np.float32),
                vec=rng.standard_normal((n, d)).astype(np.float32))


def _create(lib, h):
    import paper_2604_01960_gb300 as bbc
    s = bbc.IndexHost(h["n"], h["d"], h["L"], 0, h["M"], h["bits"], h["cent"].ctypes.data,
                      h["offs"].ctypes.data, h["ids"].ctypes.data, h["codes"].ctypes.data,
                      h["books"].ctypes.data, h["vec"].ctypes.data)
    out = C.c_void_p()
    return lib.bbc_index_create(C.byref(s), 0, C.byref(out))


def test_malformed_index_arrays_rejected_before_device(lib):
    h = _host()
    h["ids"] = h["ids"].copy(); h["ids"][3] = h["ids"][4]            # not a permutation
    assert _create(lib, h) == -3
    h = _host(); h["offs"] = h["offs"].copy(); h["offs"][-1] -= 1    # offsets do not end at n
    assert _create(lib, h) == -3
    h = _host(M=5)                                                   # pq_m does not divide d
    assert _create(lib, h) == -1
    h = _host(M=16, bits=4)                                          # 4-bit with pq_m = 16: unsupported
    assert _create(lib, h) == -9
    h = _host(d=18, M=2)                                             # d not a multiple of 4
    assert _create(lib, h) == -1


def test_index_file_writer_header(tmp_path):
    """The Python writer produces the header the C loader parses (checked field by field)."""
    import struct
    from synth.index import write_index, HEADER_FMT, IvfPqIndex
    h = _host()
    idx = IvfPqIndex("l2", h["d"], h["L"], h["M"], h["bits"], h["cent"], h["offs"], h["ids"], h["codes"],
                     h["books"], h["vec"])
    p = tmp_path / "i.bin"
    write_index(str(p), idx)
    raw = p.read_bytes()
    magic, ver, quant, metric, d, n, nlist, m, bits = struct.unpack_from(HEADER_FMT, raw)
    assert (magic, ver, quant, metric, d, n, nlist, m, bits) == (b"BBCIDX01", 1, 0, 0, 16, 64, 4, 8, 8)
    assert len(raw) >= 64 + h["cent"].nbytes + h["vec"].nbytes
