"""Host-side checks of the batched scenes: the seeded workload generator and the C ABI's
argument validation (returned before any device work, so no GPU is needed)."""
import ctypes as C

import numpy as np
import pytest

from paper_2009_14514_gb300 import rts, scenes


def test_batch_counts_are_seeded_log_uniform():
    c = scenes.batch_counts(64, seed=4321)
    assert np.array_equal(c, scenes.batch_counts(64, seed=4321))
    assert c.min() >= 10_000 and c.max() <= 200_000
    # log-uniform: the log-counts spread over the whole interval, median near the middle
    lg = np.log(c)
    assert lg.min() < np.log(1.5e4) and lg.max() > np.log(1.3e5)
    assert abs(np.median(lg) - 0.5 * (np.log(1e4) + np.log(2e5))) < 0.5


def test_batch_members_follow_their_recipe():
    b = scenes.pcisph_batch()
    assert len(b.scenes) == 64
    targets = scenes.batch_counts(64, seed=4321)
    for i, (sc, n) in enumerate(zip(b.scenes, targets)):
        if i % 2 == 0:
            c = int(np.ceil(n ** (1 / 3) - 1e-9))
            assert sc.n == c ** 3
            assert np.allclose(sc.box, (4 * c * 0.01, 2 * c * 0.01, 2 * c * 0.01))
        else:
            assert abs(sc.n / n - 1) < 0.15
        # every particle inside its own tank; every scene's grid covers its shell
        assert (sc.x >= 0).all() and (sc.x <= np.asarray(sc.box, np.float32)).all()
        o = np.asarray(sc.params["domain_min"])
        top = o + np.asarray(sc.params["grid_dim"]) * sc.params["block_edge"]
        assert (sc.xb > o).all() and (sc.xb < top).all()
    assert b.n == sum(sc.n for sc in b.scenes) and b.nb == sum(sc.nb for sc in b.scenes)
    assert [d["n_fluid"] for d in b.desc] == [sc.n for sc in b.scenes]


def test_make_batch_rejects_scenes_with_other_physics():
    a = scenes.batch_member(0, 1728)
    bad = scenes.batch_member(1, 600)
    bad.params = dict(bad.params, eta=0.02)
    with pytest.raises(ValueError):
        scenes.make_batch([a, bad])


def _init(params, desc, x, v, xb):
    P = rts.make_params(params)
    arr = (rts.RtsScene * max(len(desc), 1))()
    for k, d in enumerate(desc):
        arr[k].n_fluid = d["n_fluid"]
        arr[k].n_boundary = d["n_boundary"]
        for a in range(3):
            arr[k].domain_min[a] = d["domain_min"][a]
            arr[k].grid_dim[a] = d["grid_dim"][a]
            arr[k].wall_lo[a] = d["wall_lo"][a]
            arr[k].wall_hi[a] = d["wall_hi"][a]
    h = C.c_void_p()
    st = rts.lib().rts_batch_init(C.byref(P), len(desc), arr, x.ctypes.data, v.ctypes.data,
                                  xb.ctypes.data, None, C.byref(h))
    return st, rts.lib().rts_last_error(None).decode()


def test_batch_init_validates_arguments_on_the_host():
    b = scenes.pcisph_batch_small()
    cases = [
        (dict(b.params, scheme=scenes.WCSPH), b.desc, "RTS_PCISPH"),
        (dict(b.params, mode=scenes.MODE_GLOBAL_ADAPTIVE), b.desc, "REGIONAL"),
        (b.params, [], "n_scenes"),
        (b.params, [dict(b.desc[0], grid_dim=[0, 5, 5])] + b.desc[1:], "grid_dim"),
        (b.params, [dict(b.desc[0], wall_hi=[0.0, 0.0, 0.0])] + b.desc[1:], "wall_lo"),
        (b.params, [dict(b.desc[0], n_fluid=-1)] + b.desc[1:], "negative"),
    ]
    for params, desc, word in cases:
        st, msg = _init(params, desc, b.x, b.v, b.xb)
        assert st == 1 and word in msg, (st, msg)


def test_batch_scene_calls_reject_a_plain_context_handle():
    L = rts.lib()
    info = rts.RtsPcisphInfo()
    assert L.rts_batch_scene_info(None, 0, C.byref(info)) == 1
    assert L.rts_batch_layout(None, None, None, None, None) == 1
    assert L.rts_batch_set_launch(None, 256, 128, 1) == 1
    assert L.rts_batch_autotune(None, 1, None, None, None) == 1
