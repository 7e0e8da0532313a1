"""The tuning cache read back from its file (csrc/lattices.cu, driven on the host by
tests/tune_cache_harness.cu): well-formed lines of both kinds are found, a value outside a
kind's candidates (block sizes 64/128/256; right-hand sides per thread 1/2/4) or a malformed
line is ignored, a stored value is found again and appended in the same format, and the
right-hand-side keys name their GPU, precisions, link format, lattice and batch size.
Needs nvcc (no GPU)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))

LAT_KEY = '{"gpu":"X","sm":103,"mode":1,"lattices":[[8,8,8,8,4]]}'
RHS_KEY = '{"gpu":"X","sm":103,"what":"rhs_block","inner":2,"links":12,"outer":3,"dims":[8,6,4,6],"nrhs":8}'
BAD_BLOCK = '{"gpu":"X","sm":103,"mode":2,"lattices":[]}'
BAD_RHS = '{"gpu":"X","sm":103,"what":"rhs_block","nrhs":4}'
BAD_RHS_BLOCK = '{"gpu":"X","sm":103,"what":"rhs_block","nrhs":2}'
CUT = '{"gpu":"X","sm":103,"mode":3'


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("tune") / "tune_cache_harness")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-O1", os.path.join(HERE, "tune_cache_harness.cu"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


def _run(exe, cache, commands):
    env = dict(os.environ, LQ_TUNE_CACHE=str(cache))
    out = subprocess.run([exe], input="\n".join(commands) + "\n", capture_output=True, text=True, env=env,
                         timeout=60)
    assert out.returncode == 0, out.stderr
    return out.stdout.splitlines()


def test_cache_file_read_back(harness, tmp_path):
    cache = tmp_path / "tune.jsonl"
    cache.write_text("\n".join([
        '{"block": 128, "key": %s}' % LAT_KEY,
        '{"block": 2, "key": %s}' % RHS_KEY,
        '{"block": 100, "key": %s}' % BAD_BLOCK,
        '{"block": 3, "key": %s}' % BAD_RHS,
        '{"block": 64, "key": %s}' % BAD_RHS_BLOCK,
        'not a cache line',
        '{"block": 64, "key": %s' % CUT,
    ]) + "\n")
    got = _run(harness, cache, ["get " + k for k in (LAT_KEY, RHS_KEY, BAD_BLOCK, BAD_RHS, BAD_RHS_BLOCK, CUT)])
    assert got == ["128", "2", "none", "none", "none", "none"]


def test_store_appends_and_is_found(harness, tmp_path):
    cache = tmp_path / "tune.jsonl"
    key = RHS_KEY.replace('"nrhs":8', '"nrhs":4')
    got = _run(harness, cache, ["get " + key, "put 4 " + key, "get " + key])
    assert got == ["none", "stored", "4"]
    assert cache.read_text() == '{"block": 4, "key": %s}\n' % key
    # a new process reads it back from the file
    assert _run(harness, cache, ["get " + key]) == ["4"]


def test_right_hand_side_key(harness, tmp_path):
    key = _run(harness, tmp_path / "none.jsonl", ["rhskey"])[0]
    assert key.startswith('{"gpu":"') and key.endswith("}")
    assert '"what":"rhs_block","inner":2,"links":12,"outer":3,"dims":[8,6,4,6],"nrhs":8}' in key
