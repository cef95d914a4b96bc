"""The range-checked build (SGE_CHECKED=1, libsge_checked.so), the stand-in for a memory checker:
host-made bad inputs (bounds lowered below what the call needs, an out-of-range vertex index)
make the checks skip the access and record SGE_ERR_BOUNDS; nothing traps, the context stays
usable, and a valid call afterwards gives status 0 and the same counts."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def observed():
    from paper_2404_09758_gb300 import _build
    _build.build(checked=True)
    env = dict(os.environ, SGE_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_library_is_loaded_and_valid_calls_raise_nothing(observed):
    from paper_2404_09758_gb300 import OK
    assert observed["checked"] is True
    assert observed["parity_status"] == OK and observed["clean_status"] == OK


@pytest.mark.parametrize("name", ["vertices", "uvs", "bin_entries", "sign_words", "params"])
def test_lowered_bound_fires_then_restores(name, observed):
    from paper_2404_09758_gb300 import ERR_BOUNDS, OK
    o = observed[name]
    assert o["status"] == ERR_BOUNDS
    if name != "sign_words":  # the plain path hashes its signs: no planes to check
        assert o["plain_status"] == ERR_BOUNDS
    assert o["status_after_restore"] == OK
    assert o["counts_same_after_restore"]
    assert o["sums_rel_diff_after_restore"] < 1e-5


def test_limit_above_true_size_is_rejected(observed):
    from paper_2404_09758_gb300._abi import ERR_INVALID_ARG
    assert observed["limit_above_true_size"] == ERR_INVALID_ARG


def test_out_of_range_vertex_index_is_caught_on_every_path(observed):
    from paper_2404_09758_gb300 import ERR_BAD_INDEX, ERR_BOUNDS, OK
    assert observed["bad_index_estimate"] == ERR_BOUNDS
    assert observed["bad_index_plain"] == ERR_BOUNDS
    assert observed["bad_index_render"] == ERR_BOUNDS
    assert observed["bad_index_static"] == [OK, ERR_BOUNDS]
    assert observed["bad_index_validate"] == ERR_BAD_INDEX


def test_transparent_estimator_checks(observed):
    from paper_2404_09758_gb300 import ERR_BOUNDS, OK
    assert observed["transparent_sign_words"] == ERR_BOUNDS
    assert observed["transparent_params"] == ERR_BOUNDS
    assert observed["transparent_clean"] == OK
