"""Batched form (pilot_align_solve_batch): uneven frames x hypotheses x iterations in one
persistent launch per level, replayed from a CUDA graph.

Its reductions follow exactly the plain form's order, so every frame's outputs must be
bitwise those of its own pilot_align_solve (which is itself checked against the FP64
oracle in test_gpu_parity.py), whatever else is in the batch.
"""
import numpy as np
import pytest

from paper_2606_31098_gb300 import binding as B
from paper_2606_31098_gb300 import scenes as S

from gpu_support import require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def uneven_frames(sides=(40, 55, 70, 30), hyps=(3, 7, 5, 2), base=800):
    return [S.make_frame(S.config_reduced_frame(crop_side=s, n_hyps=m), S.frame_seed(3, base + i))
            for i, (s, m) in enumerate(zip(sides, hyps))]


def args_for(frames, dt=B.F32):
    return [B.FrameArgs(f, B.quantized_device_arrays(f, dt), is_device=True, dtype=dt) for f in frames]


def assert_same(a, b, what=""):
    np.testing.assert_array_equal(a.T_cw, b.T_cw, err_msg=what)
    np.testing.assert_array_equal(a.cost, b.cost, err_msg=what)
    np.testing.assert_array_equal(a.n_valid, b.n_valid, err_msg=what)
    np.testing.assert_array_equal(a.status, b.status, err_msg=what)
    assert a.best == b.best and a.hyp_iters == b.hyp_iters, what


@pytest.mark.parametrize("opts", [B.Options(), B.Options(iters=(4, 3, 5, 0), keep_top_k=(0, 2, 3, 0)),
                                  B.Options(damping_mode=1, lambda0=1e-2, iters=(3, 3, 3, 0))])
def test_batch_equals_each_frames_plain_solve(torch, opts):
    frames = uneven_frames()
    fas = args_for(frames)
    solver = B.Solver(opts)
    batch = solver.solve_batch(fas)
    for i, fa in enumerate(fas):
        assert_same(batch[i], solver.solve(fa), what=f"frame {i}")


def test_frame_alone_equals_frame_in_the_mix(torch):
    frames = uneven_frames(sides=(64, 33, 48), hyps=(4, 6, 3), base=900)
    fas = args_for(frames)
    solver = B.Solver(B.Options())
    mix = solver.solve_batch(fas)
    alone = solver.solve_batch([fas[1]])[0]
    assert_same(mix[1], alone)
    again = solver.solve_batch([fas[2], fas[0], fas[1]])
    assert_same(again[2], alone)
    assert_same(again[1], mix[0])


@pytest.mark.parametrize("dt", [B.BF16, B.FP8E4M3])
def test_reduced_precision_batch_equals_plain(torch, dt):
    frames = uneven_frames(sides=(50, 36), hyps=(4, 5), base=950)
    fas = args_for(frames, dt)
    solver = B.Solver(B.Options())
    batch = solver.solve_batch(fas)
    for i, fa in enumerate(fas):
        assert_same(batch[i], solver.solve(fa), what=f"frame {i}")


def test_graph_replay_with_new_frames_and_sizes(torch):
    solver = B.Solver(B.Options())
    first = args_for(uneven_frames(sides=(30, 40), hyps=(2, 3), base=970))
    solver.solve_batch(first)
    second = args_for(uneven_frames(sides=(60, 25, 45), hyps=(5, 1, 4), base=980))
    batch = solver.solve_batch(second)
    for i, fa in enumerate(second):
        assert_same(batch[i], solver.solve(fa), what=f"frame {i}")


def test_full_size_uneven_batch(torch):
    """Crops of 128^2 .. 384^2 anchors, 16-144 hypotheses, BF16 storage (the batched
    workload's shape, fewer frames): equal to the plain solve of every frame."""
    cfgs = [(128, 16), (384, 40), (192, 144), (256, 64)]
    frames = [S.make_frame(S.SceneConfig(crop_side=s, n_hyps=m), S.frame_seed(3, 1000 + i))
              for i, (s, m) in enumerate(cfgs)]
    fas = args_for(frames, B.BF16)
    solver = B.Solver(B.Options(max_points=384 * 384, max_hyps=512))
    batch = solver.solve_batch(fas)
    for i, fa in enumerate(fas):
        assert_same(batch[i], solver.solve(fa), what=f"frame {i}")
        assert batch[i].best >= 0
        er, et = S.rotation_error_deg(batch[i].T_cw[batch[i].best], frames[i].T_gt), \
            S.translation_error_m(batch[i].T_cw[batch[i].best], frames[i].T_gt)
        assert er < 0.2 and et < 1.0, (i, er, et)


def test_barrier_free_and_lockstep_levels_in_one_batch(torch):
    """Two frames of 60^2 anchors with 1200 hypotheses each: the coarse level's 8.6 M anchor x
    hypothesis units per iteration take the schedule without grid barriers, and after the
    top-8 pruning the finer levels (3600 anchors per job, under one 4096-anchor work item) run
    in lockstep; the iteration counts differ per level.  Every frame's outputs equal its plain
    solve bitwise."""
    frames = [S.make_frame(S.SceneConfig(crop_side=60, n_hyps=1200), S.frame_seed(3, 1050 + i)) for i in range(2)]
    fas = args_for(frames, B.BF16)
    opts = B.Options(max_points=60 * 60, max_hyps=2400, iters=(3, 4, 2, 0), keep_top_k=(0, 8, 8, 0))
    solver = B.Solver(opts)
    batch = solver.solve_batch(fas)
    for i, fa in enumerate(fas):
        assert_same(batch[i], solver.solve(fa), what=f"frame {i}")
    solver.close()


def test_batched_crop_sizes_bf16_against_the_oracle(torch):
    """One BF16 frame of each crop size of the batched workload (128^2, 192^2, 256^2,
    384^2 anchors, C = 32, 3 levels, priors on), solved together in one batch and checked
    against the FP64 oracle fed the dequantised maps (the values the solver uses): statuses
    equal, converged hypotheses and the selected pose within 1e-3 deg / 1 mm.  16
    hypotheses per frame keep the oracle's run to seconds."""
    from oracle import oracle as O
    from gpu_support import assert_selection_agrees, assert_solutions_agree, to_oracle_opts
    from precision_support import BF16, dequantize
    frames = [S.make_frame(S.SceneConfig(crop_side=s_, n_hyps=16), S.frame_seed(3, 1100 + i))
              for i, s_ in enumerate((128, 192, 256, 384))]
    opts = B.Options(max_points=384 * 384, max_hyps=64)
    solver = B.Solver(opts)
    fas, deq = [], []
    for f in frames:
        arrs = B.quantized_device_arrays(f, B.BF16)
        fas.append(B.FrameArgs(f, arrs, is_device=True, dtype=B.BF16))
        deq.append(f.replace(qry_feat=[dequantize(q, None, BF16).reshape(q.shape) for q in arrs["qry_feat"]],
                             ref_feat=[dequantize(r, None, BF16).reshape(r.shape) for r in arrs["ref_feat"]]))
    batch = solver.solve_batch(fas)
    solver.close()
    for i, (fd, g) in enumerate(zip(deq, batch)):
        o = O.solve(fd, to_oracle_opts(opts), n_threads=0)
        n = assert_solutions_agree(fd, opts, g, o, min_converged=4)
        assert_selection_agrees(fd, opts, g, o)
        print(f"crop {fd.N} anchors: {n} of 16 converged, all within tolerance")


def test_batch_validation(torch):
    frames = uneven_frames(sides=(20, 20), hyps=(2, 2), base=990)
    solver = B.Solver(B.Options())
    a = args_for(frames[:1])[0]
    host = B.FrameArgs(frames[1], B.host_arrays(frames[1]), is_device=False)
    with pytest.raises(B.PilotError, match="device frames"):
        solver.solve_batch([a, host])
    other = S.make_frame(S.config_reduced_frame(crop_side=20, n_hyps=2, channels=16), 5)
    with pytest.raises(B.PilotError, match="C, L and feat_dtype"):
        solver.solve_batch([a, args_for([other])[0]])
    with pytest.raises(B.PilotError, match="max_frames"):
        B.Solver(B.Options(max_frames=1)).solve_batch([a, a])
    assert solver.solve_batch([]) == []


def test_barrier_timeout_is_reported_and_the_handle_stays_usable(torch):
    """Failure detection without a fault: the level kernel's grid barrier waits are bounded
    in time.  The self-test launches that kernel with a barrier that cannot complete; every
    CTA must give up after the timeout, report it, and leave the context and the handle
    usable (a batched solve afterwards still equals the plain solves)."""
    solver = B.Solver(B.Options())
    ms = solver.selftest_barrier_timeout(100.0)
    assert 90.0 <= ms < 5000.0
    fas = args_for(uneven_frames(sides=(30, 44), hyps=(3, 2), base=1650))
    batch = solver.solve_batch(fas)
    for i, fa in enumerate(fas):
        assert_same(batch[i], solver.solve(fa), what=f"frame {i}")
    with pytest.raises(B.PilotError, match="timeout_ms"):
        solver.selftest_barrier_timeout(0.5)


def test_flag_wait_timeout_is_reported_and_the_handle_stays_usable(torch):
    """Failure detection without a fault in the schedule without grid barriers: the waits for
    a job tile's published iteration are bounded in time.  The self-test solves real frames
    (70^2 and 72^2 anchors: over 4096 anchors per job, so that schedule) with flags that can
    never be published; the first waiting CTA gives up after the timeout, the solve reports it,
    and the handle stays usable (a batched solve afterwards still equals the plain solves)."""
    fas = args_for(uneven_frames(sides=(70, 72), hyps=(4, 5), base=1660))
    solver = B.Solver(B.Options())
    ms = solver.selftest_flag_timeout(fas, 100.0)
    assert 90.0 <= ms < 5000.0
    batch = solver.solve_batch(fas)
    for i, fa in enumerate(fas):
        assert_same(batch[i], solver.solve(fa), what=f"frame {i}")
    small = args_for(uneven_frames(sides=(30,), hyps=(2,), base=1670))
    with pytest.raises(B.PilotError, match="without grid barriers"):
        solver.selftest_flag_timeout(small, 100.0)
    with pytest.raises(B.PilotError, match="timeout_ms"):
        solver.selftest_flag_timeout(fas, 0.5)


def test_autotuner_picks_a_schedule_that_keeps_the_results(torch):
    """pilot_align_autotune times the candidate schedules on the caller's frames and keeps
    the fastest for that frame shape; solves with the tuned schedule select the same pose
    (the reduction tile only changes the summation order)."""
    frames = uneven_frames(sides=(64, 64, 64, 64), hyps=(6, 6, 6, 6), base=1600)
    fas = args_for(frames)
    solver = B.Solver(B.Options())
    default = solver.schedule(fas, batched=True)
    assert default == {"tile": 1024, "ctas_per_sm": 0, "job_order": 0, "streams": 0}
    before = solver.solve_batch(fas)
    chosen, ms = solver.autotune(fas, batched=True, reps=1)
    assert chosen["tile"] in (512, 1024, 2048, 4096) and chosen["ctas_per_sm"] in (0, 1) and ms > 0
    assert solver.schedule(fas, batched=True) == chosen
    after = solver.solve_batch(fas)
    plain_chosen, _ = solver.autotune(fas[:1], batched=False, reps=1)
    assert solver.schedule(fas[:1], batched=False) == plain_chosen
    for i, f in enumerate(frames):
        a, b = before[i], after[i]
        assert (a.best >= 0) == (b.best >= 0)
        if a.best >= 0:
            assert S.rotation_error_deg(a.T_cw[a.best], b.T_cw[b.best]) < 1e-3
            assert S.translation_error_m(a.T_cw[a.best], b.T_cw[b.best]) < 1e-3
            assert a.cost[a.best] == pytest.approx(b.cost[b.best], rel=1e-5)


def test_plain_form_concurrent_parts_give_equal_results(torch):
    """The plain form's multi-stream schedule runs the hypotheses in 1-4 parts, one launch
    per part per LM iteration on its own stream; each hypothesis' records, tickets and FP64
    step are its own, so every split (uneven ones included, with top-K between levels)
    gives bitwise the one-launch results."""
    f = S.make_frame(S.config_reduced_frame(n_hyps=9), S.frame_seed(3, 1700))
    fa = args_for([f])[0]
    opts = B.Options(iters=(3, 3, 3, 0), keep_top_k=(0, 3, 7, 0))
    out = {}
    for streams in (1, 2, 3, 4):
        solver = B.Solver(opts)
        solver.set_schedule([fa], batched=False, tile=1024, streams=streams)
        out[streams] = solver.solve(fa)
        solver.close()
    for streams in (2, 3, 4):
        assert_same(out[1], out[streams], what=f"{streams} parts")


def test_roofline_probes(torch):
    """The measured ceilings bench.py compares the build pass with: positive and within the
    device's nominal rates (FP32 FMA below 2 x 128 lanes x SMs x 2.2 GHz; the gather below
    40 TB/s), and malformed maps are rejected."""
    fma = B.probe_fma()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert 0 < fma < 2 * 128 * sms * 2.2e9 / 1e12
    m = torch.zeros((64, 80, 32), dtype=torch.float32, device="cuda")
    gb = B.probe_gather(m, B.F32, 1 << 16)
    assert 0 < gb < 40000
    with pytest.raises(B.PilotError, match="tap"):
        B.probe_gather(torch.zeros((64, 80, 3), dtype=torch.float32, device="cuda"), B.F32, 1 << 10)
