"""CPU-side checks of the C-ABI library: it builds, loads, exports every entry
point include/gp.h declares, and its host-only arithmetic (the Eq. (1)-(2)
bounds) agrees with the oracle.  No compute call needs a GPU here."""
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1502_07451_b300 as gp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "gp.h")).read()
    return sorted(set(re.findall(r"^GP_API\s+[\w\s\*]+?\b(gp_\w+)\s*\(", src, flags=re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    gp.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", gp.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(gp_\w+)", out))
    names = declared()
    assert len(names) >= 20
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(gp.lib(), n)


def test_checked_library_exports_the_same_symbols():
    """libgp_checked.so (the same sources with in-kernel index tests) builds and exports every declared
    entry point; the unchecked library reports -1 for the checked word without touching a GPU."""
    from paper_1502_07451_b300 import build
    path = build.build(checked=True)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(gp_\w+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    assert gp.gp_checked_site(False) == -1


def test_bounds_match_oracle(oracle_mod):
    rng = np.random.default_rng(11)
    for _ in range(500):
        SC, SG = (int(x) for x in rng.integers(0, 2**55, 2))
        r = float(rng.choice([-1.0, 0.0, 0.25, 0.5, 1.0, rng.random()]))
        tol = float(rng.choice([0.0, 0.03, 0.1, 1.0, rng.random()]))
        assert gp.gp_bounds(SC, SG, r, tol) == oracle_mod.bounds(SC, SG, r, tol)
    for r, t in [(1.5, 0.03), (float("nan"), 0.03), (-1.0, -0.1), (-1.0, 1.5)]:
        with pytest.raises(gp.GpError) as e:
            gp.gp_bounds(10, 10, r, t)
        assert e.value.status == gp.GP_ERR_INVALID


def test_status_strings_and_families():
    assert gp.status_string(gp.GP_OK) == "ok"
    assert "cycle" in gp.status_string(gp.GP_ERR_NOT_DAG)
    fams = gp.kernel_families()
    assert "match_pick" in fams and "makespan" in fams and "contract_merge" in fams
    assert gp.gp_launch_count() >= 0


def test_library_sources_do_not_reach_the_oracle():
    """The CUDA path shares no code with the oracle and never loads it."""
    csrc = os.path.join(ROOT, "paper_1502_07451_b300")
    for dirpath, _, files in os.walk(csrc):
        for f in files:
            if f.endswith((".cu", ".cuh", ".h", ".py")):
                text = open(os.path.join(dirpath, f)).read()
                for needle in ("import oracle", "from oracle", "liboracle", "gp_oracle", "og_"):
                    assert needle not in text, (f, needle)


def test_committed_checkpoint_format_and_checksum():
    """The trained checkpoint is a version-2 file whose FNV-1a checksum (recomputed here, byte by byte)
    matches, with 37,505 finite parameters and both Adam moments."""
    import struct

    import numpy as np

    path = os.path.join(ROOT, "paper_1502_07451_b300", "models", "mpnn3_h64.bin")
    d = open(path, "rb").read()
    assert d[:8] == b"GPMPNN01"
    ver, npar = struct.unpack_from("<II", d, 8)
    assert ver == 2 and npar == 37505 and len(d) == 24 + 12 * npar + 8
    h = 0xCBF29CE484222325
    for b in d[8:-8]:
        h = ((h ^ b) * 0x100000001B3) & ((1 << 64) - 1)
    assert struct.unpack_from("<Q", d, len(d) - 8)[0] == h
    vals = np.frombuffer(d, dtype="<f4", count=3 * npar, offset=24)
    assert np.isfinite(vals).all() and (vals[2 * npar:] >= 0).all()
