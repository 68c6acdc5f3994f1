"""Host logic of bench.py: which step kernels a workload runs, the Wiener
flop model of the split DFT, per-shot cell counts with aperture windows."""
import dataclasses

import numpy as np

import bench
import lsrtm_inputs as li


def test_step_kernels_by_workload():
    w2 = li.small_case(nz=20, nx=30, nt=10, nshot=2)
    assert bench.step_kernels(w2) == {"born": "k_fwd2t", "adjoint": "k_adj2t"}
    w3 = li.small_case(ndim=3, nz=10, ny=8, nx=12, nt=10, nshot=1)
    assert bench.step_kernels(w3) == {"born": "k3f_born", "adjoint": "k3f_adj"}
    ww = dataclasses.replace(w2, geom=dataclasses.replace(
        w2.geom, win_x0=np.zeros(2, np.int32), win_nx=np.full(2, 30, np.int32)))
    assert bench.step_kernels(ww)["adjoint"] == "k_adj2d"


def test_wiener_flops_counts_the_split_dft():
    # N = 2s = 40 splits as 5 x 8: per output 13 complex multiply-adds (8 flops)
    # and one twiddle product (6 flops); 3 transforms x 2 axes x N^2 outputs
    # per block and plane, 2 planes
    nz, nx, s = 300, 2000, 20
    nk = len(range(s // 2, nz, s)) * len(range(s // 2, nx, s))
    assert bench.wiener_flops(nz, nx, s) == 2.0 * nk * 3 * 2 * 40 ** 2 * (13 * 8 + 6)
    # N = 64 = 8 x 8
    assert bench.wiener_flops(64, 64, 32) == 2.0 * 4 * 3 * 2 * 64 ** 2 * (16 * 8 + 6)


def test_shot_cells_follow_the_windows():
    w = li.small_case(nz=20, nx=30, nt=10, nshot=2, npml=5)
    assert np.allclose(bench.shot_cells(w), w.padded_cells)
    ww = dataclasses.replace(w, geom=dataclasses.replace(
        w.geom, win_x0=np.array([0, 5], np.int32), win_nx=np.array([30, 12], np.int32)))
    assert np.allclose(bench.shot_cells(ww), [(20 + 10) * (30 + 10), (20 + 10) * (12 + 10)])
