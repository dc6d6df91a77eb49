"""fgr_autotune: picks launch shapes among its candidates, leaves results
unchanged (within the FP32 tolerance), seeds later contexts of the same class,
and persists to FGR_TUNE_FILE."""

import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from workloads import random_packets

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fgr():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_21785_gb300 as pkg
    pkg.fgr.load()
    return pkg


def test_autotune_picks_candidates_and_keeps_results(fgr):
    import torch
    pk = random_packets(3, 1, 30000, q_range=(-3, 3), p_range=(-2, 2), s_range=(-1, 1))
    arrs = [torch.tensor(np.ascontiguousarray(pk[k]), dtype=torch.float64, device="cuda") for k in "qpsa"]
    packets = fgr.make_packets(*arrs)
    grid = dict(d=1, n=[8192], lo=[-math.pi], hi=[math.pi])
    with fgr.Context(1, grid, 1 / 512, fgr.make_options(precision=fgr.FGR_FP32)) as ctx:
        ref_d = torch.zeros(8192, dtype=torch.complex64, device="cuda")
        ref_f = torch.zeros_like(ref_d)
        fgr.fgr_reconstruct_direct(ctx.handle, packets, ref_d)
        fgr.fgr_reconstruct_fggc(ctx.handle, packets, ref_f)
        scratch = torch.zeros_like(ref_d)
        fgr.fgr_autotune(ctx.handle, packets, scratch, 3)
        a, b, t = fgr.fgr_get_tuning(ctx.handle)
        assert a in (2, 4, 8, 16, 32) and b in (4, 8, 16, 32, 64) and t in (32, 128)
        got_d = torch.zeros_like(ref_d)
        got_f = torch.zeros_like(ref_d)
        fgr.fgr_reconstruct_direct(ctx.handle, packets, got_d)
        fgr.fgr_reconstruct_fggc(ctx.handle, packets, got_f)
        torch.cuda.synchronize()
        for got, ref in ((got_d, ref_d), (got_f, ref_f)):
            g, r = got.cpu().numpy(), ref.cpu().numpy()
            assert np.linalg.norm(g - r) <= 1e-5 * np.linalg.norm(r)
        # a new context of the same class starts from the tuned values
        with fgr.Context(1, grid, 1 / 512, fgr.make_options(precision=fgr.FGR_FP32)) as ctx2:
            assert fgr.fgr_get_tuning(ctx2.handle) == (a, b, t)
        with pytest.raises(fgr.FgrError):
            fgr.fgr_set_tuning(ctx.handle, 0, 16)
        with pytest.raises(fgr.FgrError):
            fgr.fgr_set_tuning(ctx.handle, 4, 16, 64)
        fgr.fgr_set_tuning(ctx.handle, 3, 5, 32)
        assert fgr.fgr_get_tuning(ctx.handle) == (3, 5, 32)
        # both tile widths give the same result
        for tile in (32, 128):
            fgr.fgr_set_tuning(ctx.handle, 8, 16, tile)
            got = torch.zeros_like(ref_d)
            fgr.fgr_reconstruct_fggc(ctx.handle, packets, got)
            torch.cuda.synchronize()
            g, r = got.cpu().numpy(), ref_f.cpu().numpy()
            assert np.linalg.norm(g - r) <= 1e-5 * np.linalg.norm(r)


def test_tuning_file_persists_across_processes(tmp_path):
    path = tmp_path / "tune.txt"
    code = """
        import math, numpy as np, torch
        import paper_2504_21785_gb300 as fgr
        from workloads import random_packets
        grid = dict(d=2, n=[96, 96], lo=[-math.pi] * 2, hi=[math.pi] * 2)
        ctx = fgr.Context(2, grid, 1 / 64, fgr.make_options(precision=fgr.FGR_FP32))
        if {tune}:
            pk = random_packets(4, 2, 4000, q_range=(-1, 1), p_range=(-1, 1))
            arrs = [torch.tensor(np.ascontiguousarray(pk[k]), dtype=torch.float64, device="cuda") for k in "qpsa"]
            u = torch.zeros((96, 96), dtype=torch.complex64, device="cuda")
            fgr.fgr_autotune(ctx.handle, fgr.make_packets(*arrs), u, 1)
        print("TUNING", *fgr.fgr_get_tuning(ctx.handle))
    """
    env = dict(os.environ, FGR_TUNE_FILE=str(path), PYTHONPATH=ROOT)
    outs = []
    for tune in (True, False):
        r = subprocess.run([sys.executable, "-c", textwrap.dedent(code.format(tune=tune))], env=env, cwd=ROOT,
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        outs.append([line for line in r.stdout.splitlines() if line.startswith("TUNING")][0])
    assert path.exists() and len(path.read_text().split()) == 7
    assert outs[0] == outs[1]
