"""Continuous-batching serving loop: requests of different sizes, step
counts and precisions, arriving while others run, admitted by free memory;
each result is the same (bitwise) as the request run alone."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_09713_gb300 import build

    build.build()
    from paper_1709_09713_gb300 import sbli

    sbli.lib()
    return sbli


REQS = [  # n, precision, steps, Re, Mach, amplitude, submit at tick
    ((16, 16, 16), 0, 5, 1600.0, 0.1, 1.0, 0),
    ((24, 16, 20), 1, 9, 400.0, 0.2, 0.95, 0),
    ((32, 32, 32), 0, 3, 800.0, 0.3, 1.05, 0),
    ((20, 20, 20), 1, 7, 100.0, 0.1, 1.0, 2),
    ((40, 12, 8), 0, 4, 1200.0, 0.15, 0.9, 3),
    ((5, 6, 7), 1, 6, 50.0, 0.4, 1.1, 3),
    ((36, 36, 36), 1, 2, 1600.0, 0.1, 1.0, 5),
    ((16, 16, 16), 0, 0, 1600.0, 0.1, 1.0, 6),
    ((24, 20, 16), 3, 6, 1600.0, 0.1, 1.0, 1),  # double-float arithmetic
    ((32, 16, 12), 3, 3, 300.0, 0.2, 0.97, 4),
    ((28, 20, 12), 2, 5, 900.0, 0.25, 1.02, 1),  # binary32, double-float accumulator
    ((16, 24, 20), 2, 8, 1600.0, 0.1, 1.0, 4),
]


def alone(S, n, prec, steps, Re, M, A, dt):
    g = S.Grid(n, prec, S.SBLI_FUSED, Re=Re, Mach=M)
    g.set_config(8, min(32, n[2]))
    g.init_tgv(A)
    g.step_n(steps, dt)
    out = g.get_state()
    ke, ens = g.kinetic_energy()
    g.close()
    return out, ke, ens


def test_results_same_alone_and_in_the_mix(S):
    dt = 1e-3
    srv = S.Server(256 << 20, max_slots=8)
    outs, ids, done = {}, {}, {}
    tick = 0
    while len(done) < len(REQS):
        for i, (n, prec, steps, Re, M, A, at) in enumerate(REQS):
            if at == tick and i not in ids:
                outs[i] = torch.empty((5, n[2], n[1], n[0]), dtype=torch.float64, device="cuda")
                ids[i] = srv.submit(S.request(n, prec, steps, dt, Re=Re, Mach=M, amplitude=A, result=outs[i]))
        srv.tick()
        for r in srv.poll():
            done[r.id] = r
        tick += 1
        assert tick < 100
    st = srv.stats()
    assert st.active == 0 and st.pending == 0 and st.free_bytes == st.arena_bytes
    for i, (n, prec, steps, Re, M, A, at) in enumerate(REQS):
        want, ke, ens = alone(S, n, prec, steps, Re, M, A, dt)
        assert torch.equal(outs[i], want), i
        r = done[ids[i]]
        assert r.ke == pytest.approx(ke, rel=1e-14) and r.enstrophy == pytest.approx(ens, rel=1e-14)
        assert r.t_admit >= r.t_submit and r.t_done >= r.t_admit and r.steps == steps


def test_admission_is_bounded_by_free_memory(S):
    r0 = S.request((24, 24, 24), 0, 3)
    need = S.sbli_server_request_bytes(r0)
    arena = 2 * need + need // 2  # room for two requests at a time
    srv = S.Server(arena + 4096 * 64, max_slots=16, backfill=False)
    for i in range(5):
        srv.submit(S.request((24, 24, 24), 0, 3 + i))
    peak, finished = 0, 0
    for _ in range(60):
        srv.tick()
        st = srv.stats()
        peak = max(peak, st.active)
        finished += len(srv.poll())
        if finished == 5:
            break
    assert finished == 5 and peak == 2


def test_backfill_admits_small_request_behind_large(S):
    big = S.request((48, 48, 48), 0, 4)
    small = S.request((16, 16, 16), 1, 2)
    arena = S.sbli_server_request_bytes(big) + S.sbli_server_request_bytes(small) + (1 << 20)
    srv = S.Server(arena, max_slots=4, backfill=True)
    srv.submit(big)
    srv.submit(S.request((48, 48, 48), 0, 4))  # cannot fit while the first runs
    srv.submit(small)
    srv.tick()
    st = srv.stats()
    assert st.active == 2 and st.pending == 1


def test_server_rejects_bad_requests(S):
    srv = S.Server(8 << 20, max_slots=2)
    with pytest.raises(S.SbliError) as e:
        srv.submit(S.request((256, 256, 256), 0, 1))
    assert e.value.code == S.SBLI_ENOMEM
    with pytest.raises(S.SbliError) as e:
        srv.submit(S.request((4, 8, 8), 0, 1))
    assert e.value.code == S.SBLI_EINVAL
    with pytest.raises(S.SbliError):
        srv.submit(S.request((8, 8, 8), 0, 1, dt=-1.0))
    with pytest.raises(S.SbliError) as e:
        srv.submit(S.request((8, 8, 8), 7, 1))  # unknown precision
    assert e.value.code == S.SBLI_EINVAL
    srv.close()


def test_binary32_lane_is_not_gated_by_binary64_steps(S):
    """The two precision lanes advance independently: a short binary32
    request admitted beside a long binary64 one finishes while the binary64
    one is still running, in far less time than the binary64 request needs
    for the same number of steps (a tick that advanced both lanes together
    and waited for both would hold every binary32 step to a binary64 step)."""
    srv = S.Server(1 << 30, max_slots=4)
    long_id = srv.submit(S.request((160, 160, 160), 0, 40))
    short_id = srv.submit(S.request((32, 32, 32), 1, 40))
    done, active_at_short = {}, None
    for _ in range(100000):
        srv.tick()
        for r in srv.poll():
            done[r.id] = r
            if r.id == short_id:
                active_at_short = srv.stats().active
        if len(done) == 2:
            break
    assert len(done) == 2 and active_at_short == 1
    long_r, short_r = done[long_id], done[short_id]
    per_step_long = (long_r.t_done - long_r.t_admit) / long_r.steps
    assert short_r.t_done < long_r.t_done
    assert short_r.t_done - short_r.t_admit < 0.25 * short_r.steps * per_step_long
