"""CPU-side checks of the C ABI: the library loads, exports every declared
symbol, sizes layouts as documented, rejects bad arguments before touching
the device, and its host-side Morton order matches the oracle bit for bit."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import geo_oracle as O
from paper_2003_05324_b300 import geo, inputs

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "geo.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^int\s+(geo_\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_symbol():
    names = declared_symbols()
    assert len(names) >= 12
    lib = ctypes.CDLL(geo.LIB_PATH)
    for nm in names:
        assert hasattr(lib, nm), nm


def test_struct_sizes_match_header(tmp_path):
    """The ctypes mirrors of the ABI structs have the sizes and field offsets a C
    compiler gives the declarations in include/geo.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    checks = {
        "geo_theta": geo.geo_theta, "geo_layout": geo.geo_layout, "geo_tiles": geo.geo_tiles,
        "geo_mle_opts": geo.geo_mle_opts, "geo_mle_result": geo.geo_mle_result,
        "geo_batch_item": geo.geo_batch_item,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for name, cls in checks.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "abi"
    subprocess.run([cc, "-std=c99", "-o", str(exe), str(src)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                    check=True).stdout.splitlines())
    for name, cls in checks.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)


@pytest.mark.parametrize("n,nb,band", [(1600, 200, 8), (40000, 500, 1), (1000, 96, 2), (50, 64, 1), (1, 16, 1),
                                       (129600, 720, 3)])
def test_layout_counts(n, nb, band):
    lay = geo.layout(n, nb, band)
    p = -(-n // nb)
    assert lay.p == p and lay.nb == nb and lay.band == min(band, p)
    ndp = sum(1 for j in range(p) for i in range(j, p) if i - j < lay.band)
    assert lay.n_dp_tiles == ndp
    assert lay.n_dp_tiles + lay.n_sp_tiles == p * (p + 1) // 2
    assert lay.bytes_dp >= ndp * nb * nb * 8
    assert lay.bytes_sp >= lay.n_sp_tiles * nb * nb * 4
    assert lay.pp % 64 == 0 and lay.pp >= nb
    if p > 1:
        assert lay.bytes_planes >= 7 * lay.pp ** 2 * 2 * p * (p - 1) // 2
    assert geo.layout(n, nb, band, geo.GEO_LP_FP32).bytes_planes == 0


def test_layout_rejects_bad_arguments():
    lay = geo.geo_layout()
    L = geo.lib
    assert L.geo_layout_init(0, 64, 1, 0, ctypes.byref(lay)) == -1
    assert L.geo_layout_init(100, 8, 1, 0, ctypes.byref(lay)) == -2
    assert L.geo_layout_init(100, 2048, 1, 0, ctypes.byref(lay)) == -2
    assert L.geo_layout_init(100, 64, 0, 0, ctypes.byref(lay)) == -3
    assert L.geo_layout_init(100, 64, 1, 7, ctypes.byref(lay)) == -4
    assert L.geo_layout_init(100, 64, 1, 0, None) == -5


def test_entry_points_reject_null_arguments_without_device_work():
    L = geo.lib
    t = geo.geo_tiles()   # unbound: null device buffers
    th = geo.Theta(1.0, 0.1, 0.5).c()
    assert L.geo_matern_tiles(ctypes.byref(t), None, None, th, None) == -1
    assert L.geo_potrf_mp(None, None) == -1
    assert L.geo_logdet_trsv(ctypes.byref(t), None, None, None, None, None) == -1
    assert L.geo_loglik(None, None, None, None, th, None, None, None) == -1
    assert L.geo_krige(None, None, None, None, th, None, None, 0, None, None, None) == -1
    assert L.geo_tiles_bind(None, None, None, None, None, None, None) == -1
    assert L.geo_morton_order(None, None, 3, None) == -1
    assert L.geo_mle(None, None, None, None, th, None, None, None) == -1
    nbytes = ctypes.c_size_t(0)
    assert L.geo_batch_workspace(0, None, ctypes.byref(nbytes)) == -1
    assert L.geo_batch_workspace(1, None, ctypes.byref(nbytes)) == -2
    items = (geo.geo_batch_item * 1)()
    items[0].t = ctypes.pointer(t)                 # unbound store: rejected before any device work
    assert L.geo_batch_workspace(1, items, ctypes.byref(nbytes)) == -2
    assert L.geo_batch_bind(1, items, None, 0, None) == -2
    assert L.geo_loglik_batch(1, items, None, None, None, None, None) == -3
    assert L.geo_batch_set_ctas(None, 4) == -1
    fake = ctypes.c_void_p(4096)                   # never bound: looked up only after the argument checks
    for bad in (-1, 1, geo.GEO_MIN_CTAS - 1):
        assert L.geo_batch_set_ctas(fake, bad) == -2
    assert L.geo_batch_set_ctas(fake, geo.GEO_MIN_CTAS) == -1
    assert L.geo_batch_set_ctas(fake, 0) == -1
    assert L.geo_batch_release(None) == -1
    assert L.geo_mle_default_opts(None) == -1


def test_mle_options_defaults_and_validation():
    o = geo.geo_mle_opts()
    assert geo.lib.geo_mle_default_opts(ctypes.byref(o)) == 0
    assert (o.max_evals, o.profile, o.fix_nu) == (60, 0, 0)
    assert o.xtol == 1e-3 and o.step == 0.1
    assert list(o.lo) == [1e-3, 1e-4, 0.05] and list(o.hi) == [1e2, 2.0, 3.0]
    assert ctypes.sizeof(geo.geo_mle_opts) == 104 and ctypes.sizeof(geo.geo_mle_result) == 56
    assert o.journal is None and o.journal_cap == 0 and not o.journal_len
    t = geo.geo_tiles()
    th = geo.Theta(1.0, 0.1, 0.5).c()
    r = geo.geo_mle_result()
    d = ctypes.c_void_p(8)   # never dereferenced: validation fails first
    bad = geo.geo_mle_opts()
    geo.lib.geo_mle_default_opts(ctypes.byref(bad))
    bad.max_evals = 0
    assert geo.lib.geo_mle(ctypes.byref(t), d, d, d, th, ctypes.byref(bad), ctypes.byref(r), None) == -6
    bad.max_evals, bad.lo[1] = 60, 0.0
    assert geo.lib.geo_mle(ctypes.byref(t), d, d, d, th, ctypes.byref(bad), ctypes.byref(r), None) == -6
    assert geo.lib.geo_mle(ctypes.byref(t), d, d, d, geo.Theta(-1.0, 0.1, 0.5).c(), ctypes.byref(o),
                           ctypes.byref(r), None) == -5
    assert geo.lib.geo_mle(ctypes.byref(t), d, d, d, th, ctypes.byref(o), None, None) == -7


@pytest.mark.parametrize("seed", [0, 1])
def test_morton_order_matches_oracle(seed):
    x, y = inputs.jittered_grid(23, seed=seed)
    # add exact ties and out-of-range values to exercise clamping and tie order
    x = np.concatenate([x, [0.5, 0.5, -0.1, 1.3]])
    y = np.concatenate([y, [0.25, 0.25, 0.2, 0.9]])
    got = geo.morton_order(x, y)
    want = O.morton_order(x, y)
    assert np.array_equal(got, want)


def test_timeout_and_flag_setters_validate_without_device_work():
    t = geo.geo_tiles()
    assert geo.lib.geo_tiles_set_timeout_ns(None, 0) == -1
    for bad in (1, 99_999, 10 ** 13, -1):
        assert geo.lib.geo_tiles_set_timeout_ns(ctypes.byref(t), bad) == -2
    assert geo.lib.geo_tiles_set_timeout_ns(ctypes.byref(t), 50_000_000) == 0 and t.timeout_ns == 50_000_000
    assert geo.lib.geo_tiles_set_timeout_ns(ctypes.byref(t), 0) == 0 and t.timeout_ns == 0
    assert geo.lib.geo_tiles_set_flags(ctypes.byref(t), geo.GEO_FLAG_TEST_STALL) == 0
    assert geo.lib.geo_tiles_set_flags(ctypes.byref(t), 1 << 10) == -2


def test_mle_journal_validation_without_device_work():
    t = geo.geo_tiles()
    th = geo.Theta(1.0, 0.1, 0.5).c()
    d = ctypes.c_void_p(8)   # never dereferenced: validation fails first
    r = geo.geo_mle_result()
    o = geo.geo_mle_opts()
    geo.lib.geo_mle_default_opts(ctypes.byref(o))
    rec = np.zeros((4, 4))
    n = ctypes.c_int(5)                       # more records claimed than the journal holds
    o.journal, o.journal_cap, o.journal_len = rec.ctypes.data, 4, ctypes.pointer(n)
    assert geo.lib.geo_mle(ctypes.byref(t), d, d, d, th, ctypes.byref(o), ctypes.byref(r), None) == -6
    o.journal_len = ctypes.POINTER(ctypes.c_int)()   # journal without a length
    assert geo.lib.geo_mle(ctypes.byref(t), d, d, d, th, ctypes.byref(o), ctypes.byref(r), None) == -6


def test_binding_constants_match_the_header():
    """Every #define GEO_* value of include/geo.h has the same value in the
    Python binding (the binding restates them for marshalling only)."""
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "geo.h")).read()
    found = re.findall(r"^#define (GEO_[A-Z0-9_]+) (-?\d+)(?:LL)?\b", hdr, flags=re.M)
    assert len(found) >= 17
    for name, value in found:
        assert getattr(geo, name) == int(value), name
