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


def test_batch_against_oracle(orc):
    """Every stream of a mixed batch against its own oracle, frame by frame:
    widths that take the vector and the scalar tiles, one stream joining late
    and one leaving early.  PBAS masks bit-exact after every tick and the PBAS
    model bit-exact when a stream leaves and at the end; GMM masks equal
    except at pixels whose oracle margin came within 1e-5 of a threshold, the
    GMM model within the FP32 tolerance elsewhere (Sec. 3.1, 3.2)."""
    import torch
    from paper_2002_00250_gb300 import fos
    from _helpers import close, oracle_gmm_params, oracle_pbas_params
    from test_gpu_pbas import assert_same
    sizes = [(136, 40), (67, 45), (256, 24), (64, 48)]
    n = 8
    joins, leaves = {2: 2}, {0: 6}
    data = [scene(W, H, n, seed=60 + i, n_objects=3, hole_fraction=0.05) for i, (W, H) in enumerate(sizes)]
    b = fos.Batch(len(sizes))
    slots, ref, t_of, bad = {}, {}, {}, {}

    def check_models(i):
        W, H = sizes[i]
        st = fos.decode_state(b.get_state(slots[i]))
        g, p = ref[i]
        assert_same(st.pbas, p, t_of[i] - 1)
        for name in ("w_rgb", "mu_rgb", "v_rgb", "w_d", "mu_d", "v_d"):
            good = close(st.gmm[name], getattr(g, name)).reshape(W * H, -1).all(axis=1)
            assert good[~bad[i]].all(), (i, name)

    for step in range(n):
        for i, (W, H) in enumerate(sizes):
            if i not in slots and joins.get(i, 0) == step:
                slots[i] = b.add(W, H, stream_id=300 + i)
                prm = fos.default_params(stream_id=300 + i)
                ref[i] = (orc.GMM(W, H, **oracle_gmm_params(prm)), orc.PBAS(W, H, **oracle_pbas_params(prm)))
                t_of[i] = 0
                bad[i] = np.zeros(W * H, bool)
        active = [i for i in slots if leaves.get(i, n + 1) > step]
        rgb = [torch.from_numpy(data[i][0][t_of[i]]).cuda() for i in active]
        dep = [torch.from_numpy(data[i][1][t_of[i]]).cuda() for i in active]
        mg = [torch.empty(sizes[i][::-1], dtype=torch.uint8, device="cuda") for i in active]
        mp = [torch.empty(sizes[i][::-1], dtype=torch.uint8, device="cuda") for i in active]
        b.process([slots[i] for i in active], rgb, dep, mg, mp)
        torch.cuda.synchronize()
        for k, i in enumerate(active):
            g, p = ref[i]
            t = t_of[i]
            np.testing.assert_array_equal(mp[k].cpu().numpy(), p.step(data[i][0][t], data[i][1][t]),
                                          err_msg=f"PBAS stream {i} frame {t}")
            mo, margin = g.step(data[i][0][t], data[i][1][t], want_margin=True)
            bad[i] |= (margin < 1e-5).ravel()
            np.testing.assert_array_equal(mg[k].cpu().numpy().ravel()[~bad[i]], mo.ravel()[~bad[i]],
                                          err_msg=f"GMM stream {i} frame {t}")
            t_of[i] += 1
        for i in list(slots):
            if leaves.get(i, n + 1) == step + 1:
                check_models(i)
                b.remove(slots[i])
                del slots[i]
    for i in slots:
        check_models(i)
        assert bad[i].mean() < 0.02
    b.close()
