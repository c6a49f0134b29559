"""The checked build (libgp_checked.so: every gathered index tested in-kernel, a failed test recorded
and the access skipped; the stand-in for a sanitizer, which this pool does not offer) gives the oracle's
results, identical bytes on a second run, and no failed test on valid inputs; its self-test shows a
recorded site for an out-of-range gather without the access.  Runs in a child process, which loads the
checked library (GP_LIBRARY=checked)."""
import os
import subprocess
import sys

import pytest

import paper_1502_07451_b300 as gp

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_runs_the_path_without_a_failed_index_test():
    env = dict(os.environ, GP_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_checked_run.py")], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


def test_unchecked_build_has_no_checked_word():
    assert gp.gp_checked_site(False) == -1
    with pytest.raises(gp.GpError) as e:
        gp.gp_selftest_checked()
    assert e.value.status == gp.GP_ERR_INVALID
