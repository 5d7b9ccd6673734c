"""Several frames of many streams in one call (fos_batch_process_frames_device).

With the fused model the frames after each stream's first run in one
persistent launch over all streams, tiles waiting only for their own
stream's neighbourhood of the previous frame.  Every stream must get the
bits of processing it alone, frame by frame: masks of every frame and the
exported model, for mixed sizes, different frame counts per stream and per
call (streams at frame 0 and streams mid-sequence in one call), widths that
force one-pixel tiles, propagation and conflicting forced draws; and, against
the oracle, PBAS bit-exact and GMM within the FP32 tolerance (Sec. 3.1, 3.2).
"""
import numpy as np
import pytest

from _helpers import scene

pytestmark = pytest.mark.gpu


def _data(sizes, n, seed0=40):
    return [scene(W, H, n, seed=seed0 + i) for i, (W, H) in enumerate(sizes)]


def _run(sizes, calls, shape=None, **kw):
    """calls: list of per-stream frame counts, one list per call."""
    import torch
    from paper_2002_00250_gb300 import fos
    total = [sum(c[i] for c in calls) for i in range(len(sizes))]
    data = _data(sizes, max(total))
    dev = torch.device("cuda", 0)
    b = fos.Batch(len(sizes), **kw)
    if shape:
        b.set_shape(*shape)
    slots = [b.add(W, H, stream_id=500 + i) for i, (W, H) in enumerate(sizes)]
    rgb = [torch.from_numpy(d[0]).to(dev) for d in data]
    dep = [torch.from_numpy(d[1]).to(dev) for d in data]
    mg = [torch.zeros((max(total), H, W), dtype=torch.uint8, device=dev) for W, H in sizes]
    mp = [torch.zeros_like(m) for m in mg]
    f0 = [0] * len(sizes)
    for c in calls:
        idx = [i for i in range(len(sizes)) if c[i] > 0]
        sl = lambda t: [t[i][f0[i]:f0[i] + c[i]] for i in idx]
        b.process_frames([slots[i] for i in idx], sl(rgb), sl(dep), sl(mg), sl(mp))
        for i in idx:
            f0[i] += c[i]
    torch.cuda.synchronize()
    b.sequence_status()
    for i, (W, H) in enumerate(sizes):
        seg = fos.Segmenter(W, H, stream_id=500 + i, **kw)
        seg.set_option(fos.OPT_SEQUENCE, 0)
        ag = torch.empty((total[i], H, W), dtype=torch.uint8, device=dev)
        ap = torch.empty_like(ag)
        for f in range(total[i]):
            seg.process_device(rgb[i][f], dep[i][f], ag[f], ap[f])
        torch.cuda.synchronize()
        for f in range(total[i]):
            np.testing.assert_array_equal(mg[i][f].cpu().numpy(), ag[f].cpu().numpy(), err_msg=f"gmm s{i} f{f}")
            np.testing.assert_array_equal(mp[i][f].cpu().numpy(), ap[f].cpu().numpy(), err_msg=f"pbas s{i} f{f}")
        assert np.array_equal(b.get_state(slots[i]), seg.get_state()), f"model of stream {i}"
        seg.close()
    b.close()


EVEN = [(136, 40), (64, 48), (256, 24), (96, 32), (130, 70)]


def test_frames_equal_alone_mixed_counts():
    _run(EVEN, [[5, 3, 7, 1, 4], [4, 6, 0, 3, 2], [1, 1, 1, 1, 1]])


def test_frames_ragged_width_one_pixel_tiles():
    _run(EVEN[:3] + [(67, 45)], [[4, 2, 6, 5], [3, 3, 1, 2]])


@pytest.mark.parametrize("shape", [(2, 2, 4), (2, 1, 8), (2, 4, 8)])
def test_frames_tile_shapes(shape):
    _run(EVEN, [[3, 5, 4, 2, 6], [2, 2, 2, 2, 2]], shape=shape)


@pytest.mark.parametrize("forced", [0, 3])
def test_frames_with_propagation(forced):
    _run(EVEN[:4], [[4, 6, 2, 5], [3, 1, 4, 2]], pbas_propagate=1, forced_rng=forced, N=4)


def test_frames_many_streams_two_launches():
    # more streams than one launch takes (48): two persistent launches in a call
    sizes = [(64 + 2 * (i % 5), 16 + 4 * (i % 3)) for i in range(52)]
    _run(sizes, [[2 + i % 4 for i in range(52)], [3] * 52], N=8)


def test_frames_against_oracle(orc):
    import torch
    from paper_2002_00250_gb300 import fos
    from _helpers import close, oracle_gmm_params, oracle_pbas_params
    from test_gpu_pbas import assert_same
    sizes = [(136, 40), (64, 48), (256, 24)]
    counts = [[6, 4, 8], [3, 5, 1]]
    total = [sum(c[i] for c in counts) for i in range(3)]
    data = [scene(W, H, total[i], seed=70 + i, n_objects=3, hole_fraction=0.05) for i, (W, H) in enumerate(sizes)]
    dev = torch.device("cuda", 0)
    b = fos.Batch(len(sizes))
    slots = [b.add(W, H, stream_id=600 + i) for i, (W, H) in enumerate(sizes)]
    ref = []
    for i, (W, H) in enumerate(sizes):
        prm = fos.default_params(stream_id=600 + i)
        ref.append((orc.GMM(W, H, **oracle_gmm_params(prm)), orc.PBAS(W, H, **oracle_pbas_params(prm))))
    bad = [np.zeros(W * H, bool) for W, H in sizes]
    f0 = [0, 0, 0]
    for c in counts:
        rgb = [torch.from_numpy(data[i][0][f0[i]:f0[i] + c[i]]).to(dev) for i in range(3)]
        dep = [torch.from_numpy(data[i][1][f0[i]:f0[i] + c[i]]).to(dev) for i in range(3)]
        mg = [torch.empty((c[i], H, W), dtype=torch.uint8, device=dev) for i, (W, H) in enumerate(sizes)]
        mp = [torch.empty_like(m) for m in mg]
        b.process_frames(slots, rgb, dep, mg, mp)
        torch.cuda.synchronize()
        for i in range(3):
            g, p = ref[i]
            for k in range(c[i]):
                t = f0[i] + k
                np.testing.assert_array_equal(mp[i][k].cpu().numpy(), p.step(data[i][0][t], data[i][1][t]),
                                              err_msg=f"PBAS stream {i} frame {t}")
                mo, margin = g.step(data[i][0][t], data[i][1][t], want_margin=True)
                bad[i] |= (margin < 1e-5).ravel()
                np.testing.assert_array_equal(mg[i][k].cpu().numpy().ravel()[~bad[i]], mo.ravel()[~bad[i]],
                                              err_msg=f"GMM stream {i} frame {t}")
            f0[i] += c[i]
    for i, (W, H) in enumerate(sizes):
        st = fos.decode_state(b.get_state(slots[i]))
        g, p = ref[i]
        assert_same(st.pbas, p, total[i] - 1)
        for name in ("w_rgb", "mu_rgb", "v_rgb", "w_d", "mu_d", "v_d"):
            good = close(st.gmm[name], getattr(g, name)).reshape(W * H, -1).all(axis=1)
            assert good[~bad[i]].all(), (i, name)
        assert bad[i].mean() < 0.02
    b.close()
