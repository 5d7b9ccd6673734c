"""Joint-channel PBAS variant on the GPU against the oracle: bit-exact.

Masks, samples, D, S, R, T and the gradient sums equal the oracle's after
every frame read, on ragged and vectorised sizes, with the Philox draws and
the forced draws, with the base neighbour update and with propagation, with
the pending requests applied by the flush (state read every frame) and by the
next frame's kernel (state read every 3rd frame).
"""
import numpy as np
import pytest

from _helpers import oracle_pbas_params, scene
from test_gpu_pbas import assert_same, run_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W,H,seed", [(67, 45, 1), (136, 40, 2), (130, 33, 3)])
@pytest.mark.parametrize("every", [1, 3])
def test_joint_bit_exact(orc, W, H, seed, every):
    assert run_parity(orc, W, H, 14, seed=seed, every=every, pbas_joint=1) > 0


@pytest.mark.parametrize("W,H", [(1, 1), (3, 5), (4, 1), (2, 9), (17, 13)])
def test_joint_tiny_frames(orc, W, H):
    run_parity(orc, W, H, 8, seed=W + H, pbas_joint=1)


@pytest.mark.parametrize("N", [2, 7, 31])
def test_joint_other_sample_counts(orc, N):
    run_parity(orc, 40, 12, 10, N=N, n_min=min(2, N), seed=N, pbas_joint=1)


@pytest.mark.parametrize("every", [1, 3])
@pytest.mark.parametrize("forced", [1, 2, 3])
@pytest.mark.parametrize("prop", [0, 1])
def test_joint_forced_draws(orc, forced, prop, every):
    run_parity(orc, 35, 17, 9, seed=8, every=every, forced_rng=forced, N=4, pbas_joint=1, pbas_propagate=prop)


@pytest.mark.parametrize("W,H", [(136, 40), (67, 45)])
def test_joint_with_propagation(orc, W, H):
    assert run_parity(orc, W, H, 14, seed=5, every=4, pbas_joint=1, pbas_propagate=1) > 0


def test_joint_beside_gmm(orc):
    """Both methods in one context with the joint variant (two launches per
    frame): the PBAS part matches the oracle and the GMM masks equal those of
    a GMM-only context."""
    from paper_2002_00250_gb300 import fos
    W, H, n = 96, 40, 10
    rgb, depth, _ = scene(W, H, n, seed=6, n_objects=3, hole_fraction=0.05)
    seg = fos.Segmenter(W, H, pbas_joint=1)
    g = fos.Segmenter(W, H, methods=fos.METHOD_GMM)
    p = orc.PBAS(W, H, **oracle_pbas_params(seg.params))
    for t in range(n):
        mo = p.step(rgb[t], depth[t])
        mg, mp = seg.process_host(rgb[t], depth[t])
        mg2, _ = g.process_host(rgb[t], depth[t])
        np.testing.assert_array_equal(mp, mo, err_msg=f"frame {t}")
        np.testing.assert_array_equal(mg, mg2, err_msg=f"frame {t}")
    assert_same(seg.decode_state().pbas, p, n - 1)


def test_joint_not_batched():
    from paper_2002_00250_gb300 import fos
    with pytest.raises(fos.FosError):
        fos.Batch(2, pbas_joint=1)
