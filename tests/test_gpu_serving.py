"""Serving loop: continuous batching over controllers with warm starts.

Each controller's results are the same alone and in the mix (bit for bit:
its columns are computed by the same kernel with the same inputs whatever
else runs), equal to the direct shift + warm-started solve chain, and the
admission and supersede rules hold."""
import time

import numpy as np
import pytest

from paper_2608_25666_b300 import prism_proj as pp
from paper_2608_25666_b300 import workloads

pytestmark = pytest.mark.gpu

CTRLS = {   # name: (J, H, N, dt, prec)
    "A": (12, 30, 64, 0.05, pp.PREC_FP32),
    "B": (6, 50, 500, 0.02, pp.PREC_FP32),
    "C": (14, 64, 200, 0.02, pp.PREC_TF32X3),
    "D": (7, 45, 120, 0.02, pp.PREC_BF16X3),
}
ITERS = 80


def controller_data(name, steps):
    J, H, N, dt, prec = CTRLS[name]
    data = []
    for k in range(steps):
        b = workloads.make_custom(1000 * (ord(name) - 64) + k, N, J, H, dt)
        data.append(b)
    return data


def run_server(names, steps, interleave=True):
    S = pp.Server(mem_budget_bytes=1 << 30, max_inflight=8, deadline_ms=20.0)
    projs, ids, data = {}, {}, {}
    for nm in names:
        J, H, N, dt, prec = CTRLS[nm]
        d = controller_data(nm, steps)
        P = pp.Projector(J, H, dt, d[0]["bounds"]).factor(1.0, pp.MODE_ADMM, pp.SCALE_ROWNORM, prec)
        projs[nm], data[nm] = P, d
        ids[nm] = S.add_controller(P, N, ITERS, warm=True)
    outs = {nm: [] for nm in names}
    for k in range(steps):
        tickets = []
        for nm in names:
            J, H, N, dt, prec = CTRLS[nm]
            b = data[nm][k]
            out = np.empty((N, H, J), np.float32)
            t = S.submit(ids[nm], b["q0"], b["v0"], b["xi"], out)
            if interleave:
                tickets.append((nm, t, out))
            else:
                assert S.wait(t)[0] == "done"
                outs[nm].append(out)
        for nm, t, out in tickets:
            state, lat = S.wait(t)
            assert state == "done", (nm, state)
            outs[nm].append(out)
    st = S.stats()
    S.close()
    for P in projs.values():
        P.close()
    return outs, st


def test_same_alone_and_in_the_mix():
    alone, _ = run_server(["A"], 3)
    mix, st = run_server(["B", "A", "C", "D"], 3)
    for k in range(3):
        assert np.array_equal(alone["A"][k], mix["A"][k]), k
    assert st["completed"] == 12 and st["dropped"] == 0 and st["failed"] == 0


@pytest.mark.parametrize("name", ["C", "D"])
def test_server_equals_direct_warm_chain(name):
    import torch
    outs, _ = run_server([name], 3, interleave=False)
    J, H, N, dt, prec = CTRLS[name]
    d = controller_data(name, 3)
    P = pp.Projector(J, H, dt, d[0]["bounds"]).factor(1.0, pp.MODE_ADMM, pp.SCALE_ROWNORM, prec)
    state = None
    for k in range(3):
        xi = torch.from_numpy(d[k]["xi"]).cuda()
        q0 = torch.from_numpy(d[k]["q0"]).cuda()
        v0 = torch.from_numpy(d[k]["v0"]).cuda()
        if state is not None:
            P.shift_state(1, dual=state)
        x, _, _, new_state = P.solve_ex(q0, v0, xi, ITERS, dual_init=state, want_dual_out=True)
        state = new_state
        torch.cuda.synchronize()
        assert np.array_equal(x.cpu().numpy(), outs[name][k]), k
    P.close()


def test_admission_and_supersede():
    J, H, N, dt, prec = CTRLS["B"]
    P = pp.Projector(J, H, dt, workloads.base_bounds(J)).factor(1.0)
    small = pp.Server(mem_budget_bytes=1 << 20, max_inflight=2)
    with pytest.raises(pp.PrismError) as e:
        small.add_controller(P, 4000, ITERS)
    assert e.value.status == 5
    small.close()
    S = pp.Server(mem_budget_bytes=1 << 28, max_inflight=1)
    cid = S.add_controller(P, N, 100000, warm=True)     # tens of ms or more per request
    b = workloads.make_custom(5, N, J, H, dt)
    outs = [np.empty((N, H, J), np.float32) for _ in range(3)]
    t0 = S.submit(cid, b["q0"], b["v0"], b["xi"], outs[0])
    time.sleep(0.02)                        # t0 has been launched and is still running
    t1 = S.submit(cid, b["q0"], b["v0"], b["xi"], outs[1])
    t2 = S.submit(cid, b["q0"], b["v0"], b["xi"], outs[2])
    states = [S.wait(t0)[0], S.wait(t1)[0], S.wait(t2)[0]]
    # while the first runs, the second waits for the controller and is
    # superseded by the third (an MPC step whose successor has arrived is stale)
    assert states == ["done", "dropped", "done"], states
    st = S.stats()
    assert st["completed"] + st["dropped"] == 3
    S.close()
    P.close()


def test_timed_out_request_is_failed_and_next_starts_cold():
    """A request whose solve left the handle's timeout flag set is reported
    failed (PRISM_ERR_TIMEOUT), never done; the controller's next request
    starts from a zero multiplier.  The flag is written from the host (what a
    bounded device-side wait that ran out leaves behind): no device fault."""
    import torch
    J, H, N, dt, prec = CTRLS["C"]
    d = controller_data("C", 3)
    P = pp.Projector(J, H, dt, d[0]["bounds"]).factor(1.0, pp.MODE_ADMM, pp.SCALE_ROWNORM, prec)
    S = pp.Server(mem_budget_bytes=1 << 28, max_inflight=2)
    cid = S.add_controller(P, N, ITERS, warm=True)
    out0 = np.empty((N, H, J), np.float32)
    assert S.wait(S.submit(cid, d[0]["q0"], d[0]["v0"], d[0]["xi"], out0))[0] == "done"
    pp.test_set_device_flag(P, 1)
    out1 = np.empty((N, H, J), np.float32)
    t1 = S.submit(cid, d[1]["q0"], d[1]["v0"], d[1]["xi"], out1)
    with pytest.raises(pp.PrismError) as e:
        S.wait(t1)
    assert e.value.status == 8          # PRISM_ERR_TIMEOUT
    out2 = np.empty((N, H, J), np.float32)
    assert S.wait(S.submit(cid, d[2]["q0"], d[2]["v0"], d[2]["xi"], out2))[0] == "done"
    st = S.stats()
    assert st["completed"] == 2 and st["failed"] == 1
    S.close()
    # the flag was consumed by the failed request; the third started cold
    P.device_status()
    xi = torch.from_numpy(d[2]["xi"]).cuda()
    q0 = torch.from_numpy(d[2]["q0"]).cuda()
    v0 = torch.from_numpy(d[2]["v0"]).cuda()
    x, _, _, _ = P.solve_ex(q0, v0, xi, ITERS, want_dual_out=True)
    torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), out2)
    P.close()


def test_plain_server_arm_equals_direct_plain_solves():
    """PRISM_SERVER_PLAIN: every request is the plain comparator's cold solve,
    bit for bit, whatever else the server runs."""
    import torch
    outs, st = run_server_plain(["A", "C"], 2)
    for nm in ("A", "C"):
        J, H, N, dt, prec = CTRLS[nm]
        d = controller_data(nm, 2)
        P = pp.Projector(J, H, dt, d[0]["bounds"]).factor(1.0, pp.MODE_ADMM, pp.SCALE_ROWNORM, prec)
        for k in range(2):
            xi = torch.from_numpy(d[k]["xi"]).cuda()
            q0 = torch.from_numpy(d[k]["q0"]).cuda()
            v0 = torch.from_numpy(d[k]["v0"]).cuda()
            x, _, _ = P.solve_plain(q0, v0, xi, ITERS)
            torch.cuda.synchronize()
            assert np.array_equal(x.cpu().numpy(), outs[nm][k]), (nm, k)
        P.close()
    assert st["completed"] == 4 and st["failed"] == 0


def run_server_plain(names, steps):
    S = pp.Server(mem_budget_bytes=1 << 30, max_inflight=4, deadline_ms=20.0, plain=True)
    projs, ids, data = {}, {}, {}
    for nm in names:
        J, H, N, dt, prec = CTRLS[nm]
        d = controller_data(nm, steps)
        P = pp.Projector(J, H, dt, d[0]["bounds"]).factor(1.0, pp.MODE_ADMM, pp.SCALE_ROWNORM, prec)
        projs[nm], data[nm] = P, d
        ids[nm] = S.add_controller(P, N, ITERS, warm=True)
    outs = {nm: [] for nm in names}
    for k in range(steps):
        tickets = []
        for nm in names:
            J, H, N, dt, prec = CTRLS[nm]
            out = np.empty((N, H, J), np.float32)
            tickets.append((nm, S.submit(ids[nm], data[nm][k]["q0"], data[nm][k]["v0"], data[nm][k]["xi"], out), out))
        for nm, t, out in tickets:
            assert S.wait(t)[0] == "done"
            outs[nm].append(out)
    st = S.stats()
    S.close()
    for P in projs.values():
        P.close()
    return outs, st
