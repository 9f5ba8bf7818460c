"""C-ABI checks that need no GPU: the library loads, exports every declared
symbol, and its host-side helpers agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import superop as SO

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "eamps.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mps_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mps_create", "mps_destroy", "mps_apply_1q", "mps_apply_2q", "mps_fidelity", "mps_expect",
              "mps_amplitude", "mps_bond_dims"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_2307_16870_gb300 as E
    lib = E.load()
    for n in _declared():
        assert hasattr(lib, n), n


def test_status_strings_and_defaults():
    import paper_2307_16870_gb300 as E
    assert E.mps_status_string(0) == "ok"
    assert "cap" in E.mps_status_string(7)
    o = E.mps_default_options()
    assert o.kind == E.PURE and o.strategy == E.GLOBAL and o.precision == E.TF32X3 and o.max_sweeps == 40


def test_options_struct_layout_matches_header():
    import paper_2307_16870_gb300 as E
    # int, double, long long, 9 ints -> 4 + 4(pad) + 8 + 8 + 9*4 = 60 -> 64 with tail padding
    assert ctypes.sizeof(E.MpsOptions) == 64
    assert ctypes.sizeof(E.TruncRecord) == 48
    # the library fills the struct: its last fields land where the binding reads them
    o = E.mps_default_options()
    assert (o.max_sweeps, o.log_truncations, o.vidal, o.svd_kernel, o.qr) == (40, 1, 0, E.SVD_AUTO, E.QR_MOVES | E.QR_PRECONDITION)


def test_superop_helper_matches_oracle():
    import paper_2307_16870_gb300 as E
    ks = [W.haar_unitary(4, 7, 0) @ k for k in W.depolarizing_2q_kraus(0.05)]
    assert np.abs(E.mps_superop_from_kraus(ks, 2) - SO.from_kraus(ks, 2)).max() < 1e-14
    ad = W.amplitude_damping_kraus(0.2)
    assert np.abs(E.mps_superop_from_kraus(ad, 1) - SO.from_kraus(ad, 1)).max() < 1e-15


def test_create_rejects_bad_arguments_without_touching_the_gpu():
    import paper_2307_16870_gb300 as E
    lib = E.load()
    h = ctypes.c_void_p()
    o = E.mps_default_options()
    assert lib.mps_create(ctypes.byref(h), 1, ctypes.byref(o), None) == 1      # N < 2
    o.kind = 5
    assert lib.mps_create(ctypes.byref(h), 4, ctypes.byref(o), None) == 1
    assert h.value is None
    assert lib.mps_destroy(None) == 0


def test_batch_item_layout_matches_header(tmp_path):
    """Field offsets of BatchItem against the C struct, compiled from the header."""
    import shutil
    import subprocess
    import paper_2307_16870_gb300 as E
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    fields = ["n_qubits", "n_gates", "qs", "ops_dev", "op_dim", "target", "opt", "fidelity", "max_bond", "status"]
    src = tmp_path / "off.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"eamps.h\"\nint main(void){\n" +
                   "".join(f'  printf("%zu\\n", offsetof(mps_batch_item, {f}));\n' for f in fields) +
                   '  printf("%zu\\n", sizeof(mps_batch_item));\n  return 0;\n}\n')
    exe = tmp_path / "off"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [getattr(E.BatchItem, f).offset for f in fields] + [ctypes.sizeof(E.BatchItem)]
    assert got == want


def test_batch_rejects_bad_arguments_without_touching_the_gpu():
    import paper_2307_16870_gb300 as E
    lib = E.load()
    items = (E.BatchItem * 1)()
    assert lib.mps_batch_run(items, -1, 1, None) == 1
    assert lib.mps_batch_run(None, 2, 1, None) == 1
    assert lib.mps_batch_run(items, 1, 0, None) == 1
    assert lib.mps_batch_run(items, 0, 4, None) == 0


def test_schedule_target_matches_the_oracle_schedule():
    """mps_schedule_target (host code of the library, no GPU) against the oracle's schedule for
    every strategy, along the products of a made-up sequence of truncation fidelities."""
    import paper_2307_16870_gb300 as E
    from oracle import textbook_mps as T
    rng = np.random.default_rng(3)
    for strat in (T.NAIVE, T.GLOBAL, T.NEAREST):
        for f_min in (0.9, 0.5, 0.999):
            o = T.TextbookMPS(4, f_min=f_min, n_2q=40, strategy=strat)
            for j in range(45):
                want = o.scheduled_target()
                got = E.mps_schedule_target(strat, f_min, 40, o.n_done, o.product)
                assert abs(got - want) <= 1e-15 * max(1.0, abs(want)), (strat, f_min, j, got, want)
                o.product *= 1.0 - abs(rng.normal(0.0, 3e-3))
                o.n_done += 1
    with pytest.raises(E.MpsError):
        E.mps_schedule_target(5, 0.9, 10, 0, 1.0)


def test_option_ranges_are_checked_without_touching_the_gpu():
    """mps_options.svd_kernel accepts the four layouts (AUTO, TOURNAMENT, GRAM, TOURNAMENT_UNSPLIT)
    and mps_options.qr the four bit combinations; values outside are refused with MPS_ERR_ARG
    before any device work."""
    import ctypes as C
    import paper_2307_16870_gb300 as E
    lib = E.load()
    for field, bad in (("svd_kernel", 4), ("svd_kernel", -1), ("qr", 4), ("qr", -1)):
        o = E.MpsOptions()
        lib.mps_default_options(C.byref(o))
        setattr(o, field, bad)
        h = C.c_void_p()
        assert lib.mps_create(C.byref(h), 8, C.byref(o), None) == 1, (field, bad)
    assert E.SVD_TOURNAMENT_UNSPLIT == 3 and E.QR_MOVES | E.QR_PRECONDITION == 3
