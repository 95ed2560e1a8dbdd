"""The C-ABI library builds, loads and exports every symbol its header
declares; host-side validation and tables work without a GPU.  CPU only: no
call here launches a kernel."""

import ctypes
import os

import numpy as np
import pytest

from oracle import lbm_oracle as o
from paper_1905_09554_gb300 import lbm


@pytest.fixture(scope="module")
def lib():
    return lbm.load()


def test_header_declares_the_boundary():
    names = lbm.header_functions()
    for required in ("lbm_create", "lbm_init_ligament", "lbm_step", "lbm_moments", "lbm_destroy",
                     "lbm_diag", "lbm_set_density", "lbm_get_populations", "lbm_velocities"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in lbm.header_functions():
        assert hasattr(lib, name), name
        assert name in lbm._SIGNATURES, f"binding lacks {name}"


def test_params_layout_matches(lib):
    assert lib.lbm_params_sizeof() == ctypes.sizeof(lbm.lbm_params)


def test_defaults(lib):
    p = lbm.lbm_params_default()
    assert (p.nx, p.ny, p.nz) == (32, 32, 32)
    assert p.G == -5.5 and p.tau == 1.0 and p.storage == lbm.LBM_F32 and p.rho0 == 1.0


def test_library_lattice_is_d3q19_with_textbook_weights(lib):
    """The library's own velocity table is the same set as the oracle's,
    with the same weight per velocity (order may differ)."""
    c, w = lbm.lbm_velocities()
    lib_map = {tuple(v): wi for v, wi in zip(c, w)}
    ref_map = {tuple(v): wi for v, wi in zip(o.C, o.W)}
    assert lib_map.keys() == ref_map.keys()
    for k in ref_map:
        assert lib_map[k] == pytest.approx(ref_map[k], abs=1e-17)
    # opposite pairs sit next to each other (1,2), (3,4), ...
    for a in range(1, 19, 2):
        assert tuple(-c[a]) == tuple(c[a + 1])


@pytest.mark.parametrize("field,value,msg", [
    ("nx", 0, "box sizes"), ("tau", 0.5, "tau"), ("collision", 7, "collision"),
    ("storage", 9, "storage"), ("rho0", -1.0, "rho0"), ("tile_y", 5, "tile_y"),
    ("lattice", 1, "D3Q19"), ("zchunk", -2, "zchunk"),
])
def test_create_rejects_bad_parameters_without_touching_the_gpu(lib, field, value, msg):
    p = lbm.lbm_params_default()
    setattr(p, field, value)
    st, ctx = lbm.lbm_create(p)
    assert st == lbm.LBM_EINVAL and not ctx.value
    assert msg in lbm.lbm_last_error(None)


def test_create_rejects_bad_mrt_rates(lib):
    p = lbm.lbm_params_default()
    p.collision = lbm.LBM_MRT_GUO
    p.has_rates = 1
    for k in range(19):
        p.s[k] = 1.0
    p.s[9] = 2.5
    st, _ = lbm.lbm_create(p)
    assert st == lbm.LBM_EINVAL and "rates" in lbm.lbm_last_error(None)


def test_local_reference_storage_runs_kernels_1_3_and_7_only(lib):
    for storage in (lbm.LBM_F16_LOCAL, lbm.LBM_BF16_LOCAL):
        p = lbm.lbm_params_default()
        p.storage = storage
        for kernel in (2, 4, 5):
            p.kernel = kernel
            st, ctx = lbm.lbm_create(p)
            assert st == lbm.LBM_EINVAL and not ctx.value
            assert "kernel 1, 3 or 7" in lbm.lbm_last_error(None)


def test_paired_kernel_needs_16_bit_storage_and_even_nx(lib):
    for storage, nx in ((lbm.LBM_F32, 32), (lbm.LBM_F64, 32), (lbm.LBM_F16_DEV, 33)):
        p = lbm.lbm_params_default()
        p.storage, p.nx, p.kernel = storage, nx, 7
        st, ctx = lbm.lbm_create(p)
        assert st == lbm.LBM_EINVAL and not ctx.value
        assert "kernel 7 needs 16-bit storage and nx even" in lbm.lbm_last_error(None)


def test_two_belt_force_parameters_are_validated_before_device_work(lib):
    cases = [
        dict(G2=float("nan")),
        dict(G2=-1.0, storage=lbm.LBM_F16_DEV),
        dict(G2=-1.0, kernel=3),
        dict(G2=-1.0, tile_y=4),
        dict(G2=0.0, kernel=6),
    ]
    for case in cases:
        p = lbm.lbm_params_default()
        for k, v in case.items():
            setattr(p, k, v)
        st, ctx = lbm.lbm_create(p)
        assert st == lbm.LBM_EINVAL and not ctx.value, case
        assert "G2" in lbm.lbm_last_error(None) or "two-belt" in lbm.lbm_last_error(None), case


def test_noalloc_diagnostics_reject_local_reference_storage(lib):
    """The local formats need a context's density field; refused before any
    device work."""
    st = lbm.lbm_diag_noalloc(16, lbm.LBM_F16_LOCAL, 4, 4, 8, 1.0, 1.0, 2.3, 0.1,
                              None, None, None, None, 0, None)
    assert st == lbm.LBM_EINVAL


def test_null_context_calls_fail_cleanly(lib):
    assert lbm.lbm_save(None, "x.ckpt") == lbm.LBM_EINVAL
    assert lbm.lbm_load(None, "x.ckpt") == lbm.LBM_EINVAL
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_init_ligament(None, 8.0, 0.05, 1, 2.0, 2.3, 0.1) == lbm.LBM_EINVAL
    assert lib.lbm_time(None) == -1
    lib.lbm_destroy(None)


def test_noalloc_diagnostics_reject_boxes_beyond_the_static_scratch(lib):
    """nz above LBM_NOALLOC_MAX_NZ is refused before any device work."""
    st = lbm.lbm_diag_noalloc(16, lbm.LBM_F32, 4, 4, 8193, 1.0, 1.0, 2.3, 0.1,
                              None, None, None, None, 0, None)
    assert st == lbm.LBM_EUNSUPPORTED
    st = lbm.lbm_diag_noalloc(None, lbm.LBM_F32, 4, 4, 8, 1.0, 1.0, 2.3, 0.1,
                              None, None, None, None, 0, None)
    assert st == lbm.LBM_EINVAL


def test_header_is_plain_c_and_links_from_c(lib, tmp_path):
    """include/lbm_sc.h compiles as C99 and a C program links against the
    library: the struct layout seen by C matches the library's, and a
    validation failure comes back as a status and a message (no GPU work)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "lbm_sc.h"
int main(void) {
    lbm_params p;
    lbm_ctx *ctx = (lbm_ctx *)1;
    lbm_params_default(&p);
    if ((long long)sizeof(lbm_params) != lbm_params_sizeof()) return 2;
    if (p.nx != 32 || p.storage != LBM_F32 || p.G2 != 0.0) return 3;
    p.tau = 0.25;
    if (lbm_create(&p, &ctx) != LBM_EINVAL || ctx != NULL) return 4;
    if (strstr(lbm_last_error(NULL), "tau") == NULL) return 5;
    puts("ok");
    return 0;
}
""")
    pkg = os.path.dirname(lbm.LIB_PATH)
    exe = tmp_path / "abi"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.dirname(lbm.HEADER), str(src), "-o", str(exe),
                    "-L", pkg, "-llbm_sc", f"-Wl,-rpath,{pkg}"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr)


def test_binding_argument_checks():
    """Wrong host sizes and non-CUDA / wrong-dtype tensors raise before any
    pointer reaches the library (checks that survive python -O)."""
    import torch
    a = lbm._host_array(np.ones((2, 3, 4), dtype=np.float32), 24, "x")
    assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == 24
    with pytest.raises(ValueError):
        lbm._host_array(np.ones(23), 24, "x")
    with pytest.raises(TypeError):
        lbm._device_tensor(torch.ones(24, dtype=torch.float64), 24, "x")  # CPU tensor
    with pytest.raises(TypeError):
        lbm._device_tensor([1.0] * 24, 24, "x")


def test_lattice_keywords_reach_the_params(monkeypatch):
    """Every Lattice keyword lands in its lbm_params field (captured at
    lbm_create, which is made to refuse so that no device work starts)."""
    seen = {}

    def fake_create(p):
        seen["p"] = p
        return lbm.LBM_EINVAL, None

    monkeypatch.setattr(lbm, "lbm_create", fake_create)
    rates = [0.5 + 0.05 * k for k in range(19)]
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(7, 5, 3, G=-4.0, tau=0.8, collision="mrt", rates=rates, storage="bf16l", rho0=1.5,
                    rho_ref=0.9, dev_scale=2.0, torch_buffers=False, zchunk=12, tile_y=8, kernel=3,
                    test_stall=1, G2=0.25)
    p = seen["p"]
    assert (p.nx, p.ny, p.nz) == (7, 5, 3)
    assert (p.G, p.tau, p.rho0, p.rho_ref, p.dev_scale, p.G2) == (-4.0, 0.8, 1.5, 0.9, 2.0, 0.25)
    assert p.collision == lbm.LBM_MRT_GUO and p.storage == lbm.LBM_BF16_LOCAL
    assert p.has_rates == 1 and list(p.s) == pytest.approx(rates)
    assert (p.zchunk, p.tile_y, p.kernel, p.test_stall) == (12, 8, 3, 1)
    with pytest.raises(ValueError):
        lbm.Lattice(4, 4, 4, collision="mrt", rates=[1.0] * 18, torch_buffers=False)
    with pytest.raises(ValueError):
        lbm.Lattice(4, 4, 4, storage="f8", torch_buffers=False)


def test_batch_tune_cache(monkeypatch, tmp_path):
    """Batch(tune_cache=...) tunes once and stores the pick; a second batch
    with the same boxes and physics is created with the stored launch shape
    and does not tune; other physics get their own entry.  (The library
    calls are stand-ins: no device work.)"""
    calls = {"create": [], "tune": 0}

    def fake_create(p, dims):
        calls["create"].append((p.tile_y, p.zchunk))
        return lbm.LBM_OK, ctypes.c_void_p(1)

    def fake_tune(b, trial_steps):
        calls["tune"] += 1
        return lbm.LBM_OK, {"tile_y": 16, "zchunk": 64, "ms_per_step": 0.5}

    monkeypatch.setattr(lbm, "lbm_batch_create", fake_create)
    monkeypatch.setattr(lbm, "lbm_batch_box", lambda b, i: (lbm.LBM_OK, ctypes.c_void_p(2 + i)))
    monkeypatch.setattr(lbm, "lbm_batch_tune", fake_tune)
    monkeypatch.setattr(lbm, "lbm_batch_destroy", lambda b: None)
    cache = str(tmp_path / "tune.json")
    dims = [(16, 16, 40), (24, 24, 60)]
    lbm.Batch(dims, tune_cache=cache, G=-5.5, tau=1.0).close()
    assert calls["tune"] == 1 and calls["create"][-1] == (0, 0)
    lbm.Batch(dims, tune_cache=cache, G=-5.5, tau=1.0).close()
    assert calls["tune"] == 1 and calls["create"][-1] == (16, 64)
    lbm.Batch(dims, tune_cache=cache, G=-5.5, tau=0.8).close()
    assert calls["tune"] == 2 and calls["create"][-1] == (0, 0)
    import json
    assert len(json.load(open(cache))) == 2
    # explicit launch shapes bypass the cache
    lbm.Batch(dims, tune_cache=cache, tile_y=8, zchunk=32).close()
    assert calls["tune"] == 2 and calls["create"][-1] == (8, 32)


def test_lattice_tune_cache(monkeypatch, tmp_path):
    """Lattice.tune(cache=...) tunes once per box / parameters / GPU and
    stores the pick; a lattice with the same key applies the stored shape
    through lbm_set_kernel_config without tuning.  (Stand-ins for the
    library calls: no device work.)"""
    calls = {"tune": 0, "set": []}

    def fake_tune(ctx, trial_steps):
        calls["tune"] += 1
        return lbm.LBM_OK, {"kernel": 3, "tile_y": 16, "zchunk": 24, "ms_per_step": 1.25}

    def fake_set(ctx, kernel, tile_y, zchunk):
        calls["set"].append((kernel, tile_y, zchunk))
        return lbm.LBM_OK

    monkeypatch.setattr(lbm, "lbm_tune", fake_tune)
    monkeypatch.setattr(lbm, "lbm_set_kernel_config", fake_set)

    class Stand(lbm.Lattice):
        def __init__(self, nx, ny, nz, **kw):  # no context: only what tune() reads
            self.params = lbm._params(**kw)
            self.shape = (nz, ny, nx)
            self.storage = kw.get("storage", "f32")
            self.ctx = None

        def close(self):
            pass

    cache = str(tmp_path / "tune.json")
    first = Stand(64, 32, 24, tau=1.0).tune(cache=cache)
    assert not first["cached"] and calls["tune"] == 1 and calls["set"] == []
    again = Stand(64, 32, 24, tau=1.0).tune(cache=cache)
    assert again["cached"] and calls["tune"] == 1 and calls["set"] == [(3, 16, 24)]
    Stand(64, 32, 24, tau=0.8).tune(cache=cache)  # other physics: own entry
    Stand(64, 32, 25, tau=1.0).tune(cache=cache)  # other box: own entry
    assert calls["tune"] == 3
    import json
    assert len(json.load(open(cache))) == 3


def _fnv1a64_words(data: bytes) -> int:
    """64-bit FNV-1a over little-endian 64-bit words, the byte tail one byte
    at a time (the checkpoint checksum's stated definition)."""
    h, prime, mask = 0xCBF29CE484222325, 0x100000001B3, (1 << 64) - 1
    full = len(data) // 8 * 8
    for k in range(0, full, 8):
        h = ((h ^ int.from_bytes(data[k:k + 8], "little")) * prime) & mask
    for b in data[full:]:
        h = ((h ^ b) * prime) & mask
    return h


def _checkpoint_bytes(nx, ny, nz, storage, t, G=-5.5, tau=0.9, payload_seed=0):
    import struct
    elem = {lbm.LBM_F64: 8, lbm.LBM_F32: 4}.get(storage, 2)
    n = nx * ny * nz
    pop = 19 * n * elem
    ref = 4 * n if storage >= lbm.LBM_F16_LOCAL else 0
    head = b"LBMSCKP\0" + struct.pack("<II6iq5d19dQQ", 1, 256, nx, ny, nz, storage, 0, 0, t, G, tau, 1.0, 1.0,
                                      1.0, *([1.0] * 19), pop, ref)
    assert len(head) == 256
    body = np.random.default_rng(payload_seed).integers(0, 256, pop + ref, dtype=np.uint8).tobytes()
    return head + body + _fnv1a64_words(head + body).to_bytes(8, "little")


def test_checkpoint_info_reads_and_verifies_files_without_a_gpu(lib, tmp_path):
    """A checkpoint written here from the documented layout (256-byte header,
    payload, FNV-1a checksum) is read back by the library on the host; a
    flipped byte, a truncated file, trailing bytes and a foreign file are
    refused with LBM_EIO when verifying."""
    good = _checkpoint_bytes(5, 3, 7, lbm.LBM_F32, t=1234)
    path = tmp_path / "state.ckpt"
    path.write_bytes(good)
    info = lbm.checkpoint_info(str(path))
    assert info["dims"] == (5, 3, 7) and info["storage"] == lbm.LBM_F32 and info["t"] == 1234
    assert info["G"] == -5.5 and info["tau"] == 0.9
    local = tmp_path / "local.ckpt"  # odd payload length: the checksum's byte tail
    local.write_bytes(_checkpoint_bytes(3, 3, 3, lbm.LBM_F16_LOCAL, t=7))
    assert lbm.checkpoint_info(str(local))["storage"] == lbm.LBM_F16_LOCAL
    flipped = bytearray(good)
    flipped[300] ^= 0x10
    for name, data in {"flipped": bytes(flipped), "truncated": good[:-9], "trailing": good + b"\0",
                       "foreign": b"not a checkpoint" * 20}.items():
        bad = tmp_path / name
        bad.write_bytes(data)
        st, _ = lbm.lbm_checkpoint_info(str(bad))
        assert st == lbm.LBM_EIO, name
    # the header alone is still readable without verification
    bad = tmp_path / "flipped"
    assert lbm.lbm_checkpoint_info(str(bad), verify=False)[0] == lbm.LBM_OK
    assert lbm.lbm_checkpoint_info(str(tmp_path / "missing.ckpt"))[0] == lbm.LBM_EIO
    assert lbm.lbm_checkpoint_info("")[0] == lbm.LBM_EINVAL


def test_two_belt_tables_of_the_kernel_match_the_oracle(tmp_path):
    """The E8 vectors and shell weights compiled into the two-belt kernel
    (csrc/e8.cuh, built here as host C++) are the oracle's: the same 92
    vectors and, per shell, the weights the oracle solves for exactly."""
    import shutil
    import subprocess

    from oracle import multirange as mr

    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "e8_dump.cpp"
    src.write_text(
        '#include <cstdio>\n#include "e8.cuh"\n'
        "int main() {\n"
        "  for (int k = 0; k < lbm::mr::kNE; ++k) { auto v = lbm::mr::e8(k); std::printf(\"v %d %d %d\\n\", v.x, v.y, v.z); }\n"
        "  for (int s = 0; s <= 9; ++s) std::printf(\"p %d %.17g %.17g\\n\", s, lbm::mr::p_e8(s), lbm::mr::w_d3q19(s));\n"
        "  return 0;\n}\n")
    exe = tmp_path / "e8_dump"
    csrc = os.path.join(os.path.dirname(lbm.__file__), "csrc")
    subprocess.run([cxx, "-std=c++17", "-D__host__=", "-D__device__=", "-I", csrc, str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    vecs = sorted(tuple(int(t) for t in ln.split()[1:]) for ln in out if ln.startswith("v "))
    assert vecs == sorted(tuple(int(t) for t in v) for v in mr.E8)
    exact = mr.e8_weights()
    for ln in out:
        if ln.startswith("p "):
            _, s, p, w = ln.split()
            s, p, w = int(s), float(p), float(w)
            assert p == (float(exact[s]) if s in exact else 0.0), s
            assert w == {1: 1.0 / 18.0, 2: 1.0 / 36.0}.get(s, 0.0), s


def test_lattice_and_moment_tables_of_the_kernels_match_the_oracle(tmp_path):
    """csrc/lattice.cuh built as host C++: its velocities and weights are the
    oracle's D3Q19 set, and its moment coefficients mrt_coef(k, q) are the
    oracle's MRT matrix M[k, a] for the same velocity (row order included)."""
    import shutil
    import subprocess

    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "lattice_dump.cpp"
    src.write_text(
        '#include <cstdio>\n#include "lattice.cuh"\n'
        "int main() {\n"
        "  for (int q = 0; q < lbm::Q; ++q) {\n"
        "    std::printf(\"%d %d %d %.17g\", lbm::cx(q), lbm::cy(q), lbm::cz(q), lbm::wq(q));\n"
        "    for (int k = 0; k < lbm::Q; ++k) std::printf(\" %d\", lbm::mrt_coef(k, q));\n"
        "    std::printf(\"\\n\");\n  }\n  return 0;\n}\n")
    exe = tmp_path / "lattice_dump"
    csrc = os.path.join(os.path.dirname(lbm.__file__), "csrc")
    subprocess.run([cxx, "-std=c++17", "-D__host__=", "-D__device__=", "-D__forceinline__=inline", "-I", csrc,
                    str(src), "-o", str(exe)], check=True)
    rows = [ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                check=True).stdout.splitlines()]
    assert len(rows) == 19
    oracle_index = {tuple(int(v) for v in c): a for a, c in enumerate(o.C)}
    seen = set()
    for r in rows:
        c = (int(r[0]), int(r[1]), int(r[2]))
        a = oracle_index[c]
        seen.add(a)
        assert float(r[3]) == o.W[a], c
        assert [int(v) for v in r[4:]] == [int(round(v)) for v in o.M[:, a]], c
    assert len(seen) == 19


def test_binding_constants_match_the_header():
    """Every LBM_* enumerator the header defines has the same value in the
    binding (status codes, lattice, collision, psi law, storage)."""
    import re

    text = re.sub(r"/\*.*?\*/", "", open(lbm.HEADER).read(), flags=re.S)
    found = dict((k, int(v)) for k, v in re.findall(r"\b(LBM_[A-Z0-9_]+)\s*=\s*(\d+)", text))
    assert len(found) >= 16
    for name, value in found.items():
        if name.startswith("LBM_NOALLOC"):
            continue
        assert getattr(lbm, name) == value, name
    assert lbm.STATUS_NAMES == [k for k, _ in sorted(((k, v) for k, v in found.items()
                                                      if k in lbm.STATUS_NAMES), key=lambda kv: kv[1])]


def test_params_field_offsets_match_the_header(tmp_path):
    """Field by field, the ctypes mirror of lbm_params has the C struct's
    offsets (a reordered or retyped field would pass a size check alone)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = [f[0] for f in lbm.lbm_params._fields_]
    body = "".join(f'    printf("{n} %zu\\n", offsetof(lbm_params, {n}));\n' for n in names)
    src = tmp_path / "offsets.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "lbm_sc.h"\nint main(void) {\n' + body
                   + "    return 0;\n}\n")
    exe = tmp_path / "offsets"
    subprocess.run([cc, "-std=c99", "-I", os.path.dirname(lbm.HEADER), str(src), "-o", str(exe)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for n in names:
        assert int(got[n]) == getattr(lbm.lbm_params, n).offset, n
