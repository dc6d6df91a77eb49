"""The tensor-product description of the workload meshes (workloads.mesh_axes)
lists exactly the packet positions of workloads.wkb_packets, in the index map
it states, for the kept subset of a thresholded mesh as well."""

import math

import numpy as np
import pytest

from workloads import WKB_LINEAR, WKB_TANH, mesh_axes, wkb_packets
from workloads.wkb import select_top


@pytest.mark.parametrize("d,nq,np_,fam", [(1, 8, 6, WKB_TANH), (2, 6, 4, WKB_TANH), (3, 4, 2, WKB_LINEAR)])
def test_mesh_axes_list_the_packets(d, nq, np_, fam):
    eps = 1 / 64
    pk = wkb_packets(d, eps, nq, np_, fam)
    axes, sel = mesh_axes(d, eps, nq, np_, fam)
    L = nq * np_
    assert all(ax[0].size == L and ax[1].size == L for ax in axes)
    assert np.array_equal(np.sort(sel), np.arange(L ** d))
    idx = np.array(np.unravel_index(sel, (L,) * d))
    for l in range(d):
        assert np.array_equal(axes[l][0][idx[l]], pk["q"][l])
        assert np.array_equal(axes[l][1][idx[l]], pk["p"][l])
    # q sorted within every axis (consecutive entries share windows)
    assert all(np.all(np.diff(ax[0]) >= 0) for ax in axes)


def test_workload_axes_follow_the_kept_subset():
    eps, nq, np_ = 1 / 64, 4, 2
    pk = wkb_packets(3, eps, nq, np_, WKB_LINEAR)
    mesh = pk["mesh"]
    pref = (mesh.dq * mesh.dp) ** 3 / (2 * math.pi * eps) ** 4.5
    kept = select_top(pk, pref, 1e-8, 300)
    axes, sel = mesh_axes(3, eps, nq, np_, WKB_LINEAR)
    sub = sel[kept["kept_index"]]
    idx = np.array(np.unravel_index(sub, (nq * np_,) * 3))
    for l in range(3):
        assert np.array_equal(axes[l][0][idx[l]], kept["q"][l])
        assert np.array_equal(axes[l][1][idx[l]], kept["p"][l])
