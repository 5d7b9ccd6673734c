"""PBAS on the GPU against the oracle, through the C ABI: bit-exact.

Masks, samples, D, S, R, T and the gradient sums must equal the oracle's
after every frame (memcmp-equal arrays), on ragged and vectorised frame
sizes, with the Philox draws and with the test-only forced draws.
"""
import numpy as np
import pytest

from _helpers import oracle_pbas_params, scene

pytestmark = pytest.mark.gpu


def _seg(W, H, **kw):
    from paper_2002_00250_gb300 import fos
    kw.setdefault("methods", fos.METHOD_PBAS)
    return fos.Segmenter(W, H, **kw)


def assert_same(st, p, t):
    for name in ("sv", "sg", "sD", "R", "T", "S"):
        a, b = st[name], getattr(p, name)
        if not np.array_equal(a, b):
            idx = np.argwhere(a != b)[:5]
            raise AssertionError(f"frame {t}: {name} differs at {idx.tolist()}")
    np.testing.assert_array_equal(st["gsum"], p.gsum)


def run_parity(orc, W, H, n, seed=0, every=1, **kw):
    rgb, depth, _ = scene(W, H, n, seed=seed, n_objects=3, hole_fraction=0.05)
    seg = _seg(W, H, **kw)
    p = orc.PBAS(W, H, **oracle_pbas_params(seg.params))
    fg = 0
    for t in range(n):
        mo = p.step(rgb[t], depth[t])
        _, mp = seg.process_host(rgb[t], depth[t])
        np.testing.assert_array_equal(mp, mo, err_msg=f"mask frame {t}")
        fg += int(mo.astype(bool).sum())
        if t % every == 0 or t == n - 1:
            assert_same(seg.decode_state().pbas, p, t)
    return fg


def test_bit_exact_ragged(orc):
    assert run_parity(orc, 67, 45, 15) > 0


def test_bit_exact_vector_path(orc):
    assert run_parity(orc, 136, 40, 15, seed=2) > 0


@pytest.mark.parametrize("W,H", [(1, 1), (3, 5), (4, 1), (2, 9), (17, 13)])
def test_tiny_frames(orc, W, H):
    run_parity(orc, W, H, 8, seed=W + H)


@pytest.mark.parametrize("N", [2, 7, 31])
def test_other_sample_counts(orc, N):
    run_parity(orc, 40, 12, 10, N=N, n_min=min(2, N), seed=N)


def test_forced_draws_hand_trace(orc):
    # the oracle's hand-traced 3x3 neighbour pattern, through the GPU
    rgb = np.empty((2, 3, 3, 3), np.uint8)
    rgb[0] = 50
    rgb[1] = 50
    rgb[1, ..., 0] = 60
    depth = np.zeros((2, 3, 3), np.uint16)
    seg = _seg(3, 3, N=2, forced_rng=1)
    for t in range(2):
        seg.process_host(rgb[t], depth[t])
    sv = seg.decode_state().pbas["sv"][:, 0, :].reshape(3, 3, 2)
    assert (sv[..., 1] == 60).all()
    want0 = np.full((3, 3), 50)
    for (x, y) in [(1, 0), (2, 0), (1, 1), (2, 1)]:
        want0[y, x] = 60
    np.testing.assert_array_equal(sv[..., 0], want0)


def test_forced_draws_parity(orc):
    run_parity(orc, 33, 21, 12, forced_rng=1, N=5)


def test_480p_full_run(orc):
    # 640 x 480 x 50 frames, both methods in one context via the device API
    # (the launch configuration the benchmark times); PBAS bit-exact throughout.
    import torch
    from paper_2002_00250_gb300 import fos
    W, H, n = 640, 480, 50
    rgb, depth, _ = scene(W, H, n, seed=0)
    seg = fos.Segmenter(W, H)
    d_rgb = torch.from_numpy(rgb).cuda()
    d_dep = torch.from_numpy(depth).cuda()
    mg = torch.empty((n, H, W), dtype=torch.uint8, device="cuda")
    mp = torch.empty_like(mg)
    seg.process_device(d_rgb, d_dep, mg, mp)
    torch.cuda.synchronize()
    p = orc.PBAS(W, H, **oracle_pbas_params(seg.params))
    masks = mp.cpu().numpy()
    for t in range(n):
        np.testing.assert_array_equal(masks[t], p.step(rgb[t], depth[t]), err_msg=f"frame {t}")
    assert_same(seg.decode_state().pbas, p, n - 1)
    c = seg.get_counters()
    assert c["frames"] == n and c["own_updates"] > 0 and c["neighbour_writes"] > 0


def test_pending_updates_applied_by_next_frame(orc):
    # state read back only every 4th frame: the neighbour updates of the other
    # frames are applied inside the next frame's classify pass, not by a flush
    run_parity(orc, 96, 30, 17, seed=5, every=4)


@pytest.mark.parametrize("px,ty", [(4, 2), (4, 8), (2, 4), (2, 8), (1, 8)])
def test_tile_shapes_give_identical_bits(px, ty):
    from paper_2002_00250_gb300 import fos
    W, H, n = 136, 40, 9
    rgb, depth, _ = scene(W, H, n, seed=3)
    ref = _seg(W, H)
    ref.process_host(rgb, depth)
    seg = _seg(W, H)
    seg.set_option(fos.OPT_PBAS_PX, px)
    seg.set_option(fos.OPT_PBAS_TY, ty)
    seg.process_host(rgb, depth)
    np.testing.assert_array_equal(seg.get_state(), ref.get_state())


@pytest.mark.parametrize("W,H", [(136, 40), (67, 45)])
def test_fused_gmm_pbas_launch_gives_identical_bits(W, H):
    # both methods, 3+3 model: frames >= 1 run as one fused launch; the same
    # context with the option off runs the two separate kernels
    from paper_2002_00250_gb300 import fos
    rgb, depth, _ = scene(W, H, 8, seed=17)
    a = fos.Segmenter(W, H)
    b = fos.Segmenter(W, H)
    b.set_option(fos.OPT_FUSE, 0)
    ma = a.process_host(rgb, depth)
    mb = b.process_host(rgb, depth)
    np.testing.assert_array_equal(ma[0], mb[0])
    np.testing.assert_array_equal(ma[1], mb[1])
    np.testing.assert_array_equal(a.get_state(), b.get_state())


# ---- spatial propagation: a neighbour update writes the requester's value ----

@pytest.mark.parametrize("W,H,seed", [(67, 45, 5), (136, 40, 6)])
def test_propagation_bit_exact(orc, W, H, seed):
    assert run_parity(orc, W, H, 14, seed=seed, pbas_propagate=1) > 0


def test_propagation_pending_requests(orc):
    """State read every 4th frame: the requests of the frames in between are
    applied by the next frame's kernel from the second value plane."""
    run_parity(orc, 64, 40, 13, seed=7, every=4, pbas_propagate=1)


@pytest.mark.parametrize("every", [1, 3])
@pytest.mark.parametrize("forced", [1, 2, 3])
def test_propagation_forced_draws(orc, forced, every):
    """Forced modes 2 and 3 make pixels receive two requests for the same
    slot, and mode 3 also requests for the slot of the pixel's own update:
    the kernel must apply the oracle's rule (the own update keeps its slot;
    the lowest direction index seen from the asked pixel wins), both in the
    flush before a state read (every frame) and inside the next frame's
    classify kernel (state read every 3rd frame)."""
    run_parity(orc, 35, 17, 9, seed=8, every=every, forced_rng=forced, N=4, pbas_propagate=1)


@pytest.mark.parametrize("W,H", [(136, 40), (67, 45)])
def test_propagation_forced_conflicts_fused(orc, W, H):
    """Both methods in one kernel (the fused path) with the conflict-making
    draws: the PBAS state still matches the oracle bit for bit."""
    from paper_2002_00250_gb300 import fos
    rgb, depth, _ = scene(W, H, 9, seed=9, n_objects=3, hole_fraction=0.05)
    seg = fos.Segmenter(W, H, forced_rng=3, N=4, pbas_propagate=1)
    p = orc.PBAS(W, H, **oracle_pbas_params(seg.params))
    for t in range(9):
        mo = p.step(rgb[t], depth[t])
        _, mp = seg.process_host(rgb[t], depth[t])
        np.testing.assert_array_equal(mp, mo, err_msg=f"mask frame {t}")
    assert_same(seg.decode_state().pbas, p, 8)
