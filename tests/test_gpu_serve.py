"""Serving (pilot_serve_*): continuous batching with admission by slots and device memory.

Every served frame's result must be bitwise the result of its own pilot_align_solve
(which test_gpu_parity.py ties to the FP64 oracle), whether it is served alone or while
other frames of other sizes are in flight at other pyramid levels.
"""
import time

import numpy as np
import pytest

from paper_2606_31098_gb300 import binding as B
from paper_2606_31098_gb300 import scenes as S

from gpu_support import require_cuda
from test_gpu_batch import args_for, assert_same, uneven_frames

pytestmark = pytest.mark.gpu

BUDGET = 2 << 30


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def test_served_mix_equals_plain_solves(torch):
    frames = uneven_frames(sides=(40, 55, 70, 30, 62), hyps=(3, 7, 5, 2, 4), base=1100)
    fas = args_for(frames)
    opts = B.Options()
    plain = [B.Solver(opts).solve(fa) for fa in fas]
    server = B.Server(opts, BUDGET, max_slots=8)
    tickets = [server.submit(fa) for fa in fas]
    for i, t in enumerate(tickets):
        res, lat = server.wait(t)
        assert_same(res, plain[i], what=f"frame {i}")
        assert lat > 0
    st = server.stats()
    assert st["completed"] == len(fas) and st["active"] == 0 and st["arena_bytes_in_use"] == 0
    server.close()


@pytest.mark.parametrize("levels", [2, 3, 0])
def test_several_levels_per_round_equal_plain_solves(torch, levels):
    """With several levels per round the device advances each frame between launches (top-K,
    next level, job tables); frames arriving mid-way join the next round. Outputs stay
    bitwise those of the plain solves, with pruning on.  With 0 the count is per frame: the
    256^2-anchor frame with 40 hypotheses (above 2^21 anchor x hypotheses) runs one level per
    round while the small ones run all of theirs."""
    frames = uneven_frames(sides=(40, 55, 256, 30, 62), hyps=(9, 7, 40, 5, 8), base=1150)
    fas = args_for(frames)
    opts = B.Options(iters=(3, 4, 2, 0), keep_top_k=(0, 3, 4, 0))
    plain = [B.Solver(opts).solve(fa) for fa in fas]
    server = B.Server(opts, BUDGET, max_slots=8)
    server.set_levels_per_round(levels)
    tickets = []
    for i, fa in enumerate(fas):
        tickets.append(server.submit(fa))
        if i == 2:
            time.sleep(0.003)
    for i, t in enumerate(tickets):
        res, _ = server.wait(t)
        assert_same(res, plain[i], what=f"frame {i}, {levels} levels per round")
    st = server.stats()
    assert st["completed"] == len(fas) and st["active"] == 0
    with pytest.raises(B.PilotError, match="before the first frame"):
        server.set_levels_per_round(1)
    server.close()


@pytest.mark.parametrize("reserved", [8, 100])
def test_reserved_sms_leave_results_unchanged(torch, reserved):
    """Rounds that leave CTA slots free for client work (a smaller persistent grid) give the
    plain solves' outputs bitwise, with the two-half schedule (the 256^2 frame with 130
    hypotheses is above its 2^23-unit threshold at the coarse level) and without."""
    frames = uneven_frames(sides=(40, 256, 30), hyps=(9, 130, 5), base=1170)
    fas = args_for(frames)
    opts = B.Options(iters=(3, 4, 2, 0), keep_top_k=(0, 3, 4, 0))
    plain = [B.Solver(opts).solve(fa) for fa in fas]
    server = B.Server(opts, BUDGET, max_slots=4)
    with pytest.raises(B.PilotError, match="reserved SMs"):
        server.set_reserved_sms(-1)
    server.set_reserved_sms(reserved)
    tickets = [server.submit(fa) for fa in fas]
    for i, t in enumerate(tickets):
        res, _ = server.wait(t)
        assert_same(res, plain[i], what=f"frame {i}, {reserved} SMs reserved")
    with pytest.raises(B.PilotError, match="before the first frame"):
        server.set_reserved_sms(0)
    server.close()


def test_light_and_heavy_rounds_equal_plain_solves(torch):
    """A round's work items are one anchor tile when the round is light and four tiles
    otherwise (three 256^2-anchor frames with 80 hypotheses each make 960 four-tile items, over
    twice the grid); the records and their FP64 sums do not depend on it, so every frame equals
    its plain solve bitwise either way, including a small frame served alone afterwards."""
    frames = uneven_frames(sides=(256, 256, 256, 48), hyps=(80, 80, 80, 6), base=1180)
    fas = args_for(frames, B.BF16)
    opts = B.Options(iters=(3, 3, 2, 0), keep_top_k=(0, 8, 8, 0), max_hyps=256)
    plain = [B.Solver(opts).solve(fa) for fa in fas]
    server = B.Server(opts, BUDGET, max_slots=4)
    tickets = [server.submit(fa) for fa in fas[:3]]
    for i, t in enumerate(tickets):
        assert_same(server.wait(t)[0], plain[i], what=f"frame {i} in a heavy round")
    assert_same(server.wait(server.submit(fas[3]))[0], plain[3], what="small frame alone")
    server.close()


def test_result_alone_equals_result_in_the_mix(torch):
    frames = uneven_frames(sides=(48, 66, 35), hyps=(5, 3, 6), base=1200)
    fas = args_for(frames, B.BF16)
    opts = B.Options(iters=(4, 4, 4, 0), keep_top_k=(0, 2, 4, 0))
    server = B.Server(opts, BUDGET, max_slots=4)
    alone, _ = server.wait(server.submit(fas[1]))
    # the same frame again, submitted between others while they are in flight
    t0 = server.submit(fas[0])
    time.sleep(0.002)
    t1 = server.submit(fas[1])
    t2 = server.submit(fas[2])
    mixed, _ = server.wait(t1)
    server.wait(t0)
    server.wait(t2)
    assert_same(mixed, alone)
    assert_same(mixed, B.Solver(opts).solve(fas[1]))
    server.close()


def test_admission_by_memory_serialises_frames_that_do_not_fit_together(torch):
    frames = uneven_frames(sides=(50, 50, 50), hyps=(3, 3, 3), base=1300)
    fas = args_for(frames)
    nbytes = sum(a.numel() * a.element_size() for k, v in fas[0].arrays.items()
                 for a in (v if isinstance(v, list) else [v]) if a is not None)
    one = int(1.6 * nbytes)          # room for one frame (plus alignment), not for two
    server = B.Server(B.Options(), one, max_slots=8)
    tickets = [server.submit(fa) for fa in fas]
    res = [server.wait(t)[0] for t in tickets]
    st = server.stats()
    assert st["peak_active"] == 1
    assert st["arena_bytes_peak"] <= one
    for i, fa in enumerate(fas):
        assert_same(res[i], B.Solver(B.Options()).solve(fa), what=f"frame {i}")
    server.close()


def test_host_frames_are_staged_into_the_arena(torch):
    f = S.make_frame(S.config_reduced_frame(crop_side=45, n_hyps=4), S.frame_seed(3, 1400))
    host = B.FrameArgs(f, B.host_arrays(f), is_device=False)
    server = B.Server(B.Options(), BUDGET, max_slots=2)
    res, _ = server.wait(server.submit(host))
    assert_same(res, B.Solver(B.Options()).solve(args_for([f])[0]))
    server.close()


def test_submit_errors(torch):
    fas = args_for(uneven_frames(sides=(30,), hyps=(2,), base=1500))
    server = B.Server(B.Options(), BUDGET, max_slots=1)
    server.wait(server.submit(fas[0]))
    other = S.make_frame(S.config_reduced_frame(crop_side=20, n_hyps=2, channels=16), 5)
    with pytest.raises(B.PilotError, match="share C, L"):
        server.submit(args_for([other])[0])
    tiny = B.Server(B.Options(), 1 << 20, max_slots=1)
    with pytest.raises(B.PilotError, match="budget"):
        tiny.submit(fas[0])
    # a full pending queue answers EBUSY (the worker is busy with the first frames)
    busy = 0
    tickets = []
    for _ in range(200):
        try:
            tickets.append(server.submit(fas[0]))
        except B.PilotError as e:
            assert e.status == B.PILOT_EBUSY
            busy += 1
    assert busy > 0
    for t in tickets:
        server.wait(t)
    server.close()
    tiny.close()


def test_served_stream_frames_equal_their_alone_solve(torch):
    """Serving workload frames (a device crop around the stream's estimate, grid hypotheses,
    BF16 features; serving.StreamClient.prepare) from four streams are in the server
    together; each result equals pilot_align_solve of the same frame alone, bitwise."""
    from paper_2606_31098_gb300 import serving as SV
    from paper_2606_31098_gb300 import tracking as TK
    g = S.make_global_map(side=2048, seed=31, n_hills=256, n_boxes=512)
    sc = S.StreamConfig(n_frames=4)
    net = S.StreamNetwork(sc, 5)
    dsm = torch.as_tensor(g.dsm, device="cuda")
    H0, W0 = sc.levels[0]
    cam = TK.Camera(sc.f0, sc.f0, W0 / 2.0, H0 / 2.0, W0, H0)
    server = B.Server(B.Options(max_points=384 * 384, max_hyps=4 * 144), 8 << 30, max_slots=8)
    client = SV.StreamClient(server, g, dsm, sc, net, cam)
    prepared = []
    for sid in range(4):
        gt = S.stream_trajectory(g, sc, 100 + sid)
        st = SV.StreamState(gt, S.stream_sensors(g, sc, gt, 200 + sid), np.zeros(sc.n_frames), gt[0].copy())
        prep = client.prepare(sid, st, 1)
        assert prep is not None
        prepared.append(prep)
    tickets = [server.submit(fa) for fa, _, _ in prepared]
    served = [server.wait(tk)[0] for tk in tickets]
    server.close()
    solver = B.Solver(B.Options(max_points=384 * 384, max_hyps=144))
    for (fa, origin, keep), r in zip(prepared, served):
        alone = solver.solve(fa)
        np.testing.assert_array_equal(r.T_cw, alone.T_cw)
        np.testing.assert_array_equal(r.cost, alone.cost)
        np.testing.assert_array_equal(r.status, alone.status)
        assert r.best == alone.best and r.best >= 0
    solver.close()


def test_stream_descriptors_batched_equal_one_by_one(torch):
    """The network stand-in describes the frames prepared together in one pass per pyramid;
    each frame's descriptors equal its own one-frame pass bitwise."""
    sc = S.StreamConfig(n_frames=4)
    net = S.StreamNetwork(sc, 7)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    items = []
    for k, n in enumerate((500, 1300, 64, 900)):
        pts = torch.rand((3, n), generator=gen, device="cuda") * 200.0 - 100.0
        pts[2] = pts[2] * 0.1
        T = np.eye(3, 4)
        T[:, 3] = (5.0 * k, -3.0, 250.0)
        items.append((k % 2, pts, T.ravel(), 1000 + k))
    both = net.descriptors_batch(items)
    for (b, pts, T, seed), got in zip(items, both):
        one = net.descriptors(b, pts, T, seed)
        assert len(one) == len(got) == len(sc.levels)
        for a, c in zip(one, got):
            assert a.shape == (pts.shape[1], sc.channels)
            assert torch.equal(a, c)

