"""Batched multi-stream launch vs each stream processed alone: identical bits.

Every pixel of every stream runs the same code on the same data in both
paths, so masks after every step and the exported models must be equal
(GMM included), for mixed sizes, for streams that join and leave, and for
every kernel shape the autotuner may pick.
"""
import numpy as np
import pytest

from _helpers import scene

pytestmark = pytest.mark.gpu


def _frames(sizes, n, seed0=30):
    import torch
    out = []
    for i, (W, H) in enumerate(sizes):
        rgb, depth, _ = scene(W, H, n, seed=seed0 + i)
        out.append((torch.from_numpy(rgb).cuda(), torch.from_numpy(depth).cuda()))
    return out


def _run(sizes, n, shape=None, joins=None, leaves=None, autotune=False, **kw):
    import torch
    from paper_2002_00250_gb300 import fos
    joins = joins or {}
    leaves = leaves or {}
    frames = _frames(sizes, n)
    b = fos.Batch(len(sizes), **kw)
    if shape:
        b.set_shape(*shape)
    slots = {}
    alone = {}
    t_of = {}
    masks_b, masks_a = {}, {}
    for step in range(n):
        for i, (W, H) in enumerate(sizes):
            if i not in slots and joins.get(i, 0) == step:
                slots[i] = b.add(W, H, stream_id=100 + i)
                alone[i] = fos.Segmenter(W, H, stream_id=100 + i, **kw)
                t_of[i] = 0
        active = [i for i in slots if leaves.get(i, n + 1) > step]
        if autotune and step == 1:
            b.autotune([slots[i] for i in active], [frames[i][0][t_of[i]] for i in active],
                       [frames[i][1][t_of[i]] for i in active])
        rgb = [frames[i][0][t_of[i]] for i in active]
        dep = [frames[i][1][t_of[i]] for i in active]
        mg = [torch.empty(sizes[i][::-1], dtype=torch.uint8, device="cuda") for i in active]
        mp = [torch.empty(sizes[i][::-1], dtype=torch.uint8, device="cuda") for i in active]
        b.process([slots[i] for i in active], rgb, dep, mg, mp)
        for k, i in enumerate(active):
            ag = torch.empty_like(mg[k])
            ap = torch.empty_like(mp[k])
            alone[i].process_device(rgb[k], dep[k], ag, ap)
            masks_b.setdefault(i, []).append((mg[k], mp[k]))
            masks_a.setdefault(i, []).append((ag, ap))
            t_of[i] += 1
        for i in list(slots):
            if leaves.get(i, n + 1) == step + 1:
                st_b = b.get_state(slots[i])
                np.testing.assert_array_equal(st_b, alone[i].get_state())
                b.remove(slots[i])
                del slots[i]
    torch.cuda.synchronize()
    for i in masks_b:
        for f, ((bg, bp), (ag, ap)) in enumerate(zip(masks_b[i], masks_a[i])):
            np.testing.assert_array_equal(bg.cpu().numpy(), ag.cpu().numpy(), err_msg=f"gmm s{i} f{f}")
            np.testing.assert_array_equal(bp.cpu().numpy(), ap.cpu().numpy(), err_msg=f"pbas s{i} f{f}")
    for i in slots:
        np.testing.assert_array_equal(b.get_state(slots[i]), alone[i].get_state())
    b.close()


SIZES = [(136, 40), (64, 48), (256, 24), (424, 16)]


def test_batch_equals_alone_mixed_sizes():
    _run(SIZES, 6)


def test_batch_ragged_width_uses_scalar_tiles():
    _run(SIZES + [(67, 45)], 5)


@pytest.mark.parametrize("shape", [(1, 2, 8), (2, 2, 4), (2, 4, 4), (2, 4, 8), (2, 1, 8)])
def test_batch_shapes(shape):
    _run(SIZES, 4, shape=shape)


def test_streams_join_and_leave():
    _run(SIZES, 7, joins={2: 2, 3: 4}, leaves={0: 5})


def test_autotune_keeps_results():
    _run(SIZES, 5, autotune=True)


@pytest.mark.parametrize("forced", [0, 3])
def test_batch_with_propagation(forced):
    """Spatial propagation in the batched kernel, with the Philox draws and
    with the conflict-making forced draws; streams join and leave."""
    _run(SIZES, 6, joins={2: 1}, leaves={0: 4}, pbas_propagate=1, forced_rng=forced, N=4)
