"""Solve server: requests of different sizes admitted by device footprint and
run concurrently; each result is the same alone and in the mix (P13)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1712_02443_gb300 as mm  # noqa: E402
from paper_1712_02443_gb300 import workloads as wl  # noqa: E402
from paper_1712_02443_gb300.arrays import build_types  # noqa: E402

pytestmark = pytest.mark.gpu
OUTERS = (0.30, 0.34, 0.38, 0.42)


@pytest.fixture(scope="module")
def family():
    from paper_1712_02443_gb300.build import build
    build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = mm.mm_ctx_create(0)
    base = wl.loop_array(2, 2, outers=OUTERS, config_index=2)
    meshes, types = build_types(ctx, base)
    yield types
    for t in types:
        mm.mm_type_destroy(t)
    for m in meshes:
        mm.mm_mesh_destroy(m)
    mm.mm_ctx_destroy(ctx)


def _requests():
    """Seeded mix: sides 2..4, 1..4 right-hand sides, tolerances 1e-3 / 1e-4."""
    g = wl.rng(4, 1)
    reqs = []
    for i in range(7):
        side = int(g.integers(2, 5))
        nrhs = int(g.integers(1, 5))
        lay = wl.loop_array(side, side, outers=OUTERS, config_index=2)
        type_of = g.integers(0, 4, size=side * side)
        th = g.uniform(0, np.pi / 3, nrhs)
        ph = g.uniform(0, np.pi / 2, nrhs)
        pol = g.integers(0, 2, nrhs)
        tol = 1e-4 if i % 2 == 0 else 1e-3
        reqs.append((type_of, lay.offsets, th, ph, pol, tol))
    return reqs


def _submit(sv, types, req):
    type_of, offs, th, ph, pol, tol = req
    return mm.mm_server_submit(sv, [types[t] for t in type_of], offs, th, ph, pol, tol)


def test_result_same_alone_and_in_mix(family):
    """The probe request is solved to 1e-6 alone and in a mix of seven requests
    in flight on three workers; the two solutions agree within the stated
    solution tolerance, 1e-4 (each is within cond * 1e-6 of the exact one)."""
    reqs = _requests()
    probe = 2
    reqs[probe] = reqs[probe][:5] + (1e-6,)
    sv = mm.mm_server_create(0, workers=1)
    try:
        t = _submit(sv, family, reqs[probe])
        res_alone, E_alone = mm.mm_server_poll(sv, t, wait=True, nrhs=len(reqs[probe][2]))
    finally:
        mm.mm_server_destroy(sv)
    assert res_alone["status"] == 0 and res_alone["converged"]
    sv = mm.mm_server_create(0, workers=3)
    try:
        tickets = [_submit(sv, family, q) for q in reqs]
        out = [mm.mm_server_poll(sv, tk, wait=True, nrhs=len(q[2])) for tk, q in zip(tickets, reqs)]
    finally:
        mm.mm_server_destroy(sv)
    for (res, E), q in zip(out, reqs):
        assert res["status"] == 0 and res["converged"] and res["rel_residual"] <= q[5]
        assert res["latency_s"] >= res["setup_s"] + res["solve_s"] - 1e-6
    E_mix = out[probe][1]
    assert np.linalg.norm(E_mix - E_alone) / np.linalg.norm(E_alone) <= 1e-4


def test_same_geometry_requests_are_solved_together(family):
    """Requests with the same array and options that wait while the only worker
    is busy join one solve as columns; each still gets its own solution, equal
    to its solution alone within 1e-4 (solves to 1e-6)."""
    g = wl.rng(4, 3)
    lay = wl.loop_array(3, 3, outers=OUTERS, config_index=2)
    type_of = g.integers(0, 4, size=9)
    shared = []
    for i in range(4):
        nrhs = 1 + i % 3
        shared.append((type_of, lay.offsets, g.uniform(0, np.pi / 3, nrhs), g.uniform(0, np.pi / 2, nrhs),
                       g.integers(0, 2, nrhs), 1e-6))
    alone = []
    sv = mm.mm_server_create(0, workers=1)
    try:
        for q in shared:
            t = _submit(sv, family, q)
            alone.append(mm.mm_server_poll(sv, t, wait=True, nrhs=len(q[2]))[1])
        # a larger request keeps the worker busy while the four wait in the queue
        big = wl.loop_array(6, 6, outers=OUTERS, config_index=2)
        busy = (g.integers(0, 4, size=36), big.offsets, [0.0], [0.0], [0], 1e-6)
        tb = _submit(sv, family, busy)
        tickets = [_submit(sv, family, q) for q in shared]
        out = [mm.mm_server_poll(sv, tk, wait=True, nrhs=len(q[2])) for tk, q in zip(tickets, shared)]
        mm.mm_server_poll(sv, tb, wait=True, want_solution=False)
    finally:
        mm.mm_server_destroy(sv)
    groups = [r["group_requests"] for r, _ in out]
    assert max(groups) == len(shared), groups
    assert all(r["group_columns"] == sum(len(q[2]) for q in shared) for r, _ in out)
    for (res, E), E1 in zip(out, alone):
        assert res["status"] == 0 and res["converged"]
        assert np.linalg.norm(E - E1) / np.linalg.norm(E1) <= 1e-4


def test_request_without_csr_assembly(family):
    """A request that skips the near-field CSR (aim.near_csr = 2: the complex128
    residual products use the dense blocks) gives the same solution."""
    q = _requests()[1][:5] + (1e-6,)
    outs = []
    for csr in (0, 2):
        sv = mm.mm_server_create(0, workers=1)
        try:
            type_of, offs, th, ph, pol, tol = q
            t = mm.mm_server_submit(sv, [family[k] for k in type_of], offs, th, ph, pol, tol, near_csr=csr)
            res, E = mm.mm_server_poll(sv, t, wait=True, nrhs=len(th))
            assert res["status"] == 0 and res["converged"]
            outs.append(E)
        finally:
            mm.mm_server_destroy(sv)
    assert np.linalg.norm(outs[0] - outs[1]) / np.linalg.norm(outs[0]) <= 1e-4


def test_admission_by_footprint(family):
    """A budget that fits one request at a time still completes every request."""
    reqs = _requests()[:3]
    sv = mm.mm_server_create(0, workers=3, hbm_budget_bytes=1)
    try:
        tickets = [_submit(sv, family, q) for q in reqs]
        out = [mm.mm_server_poll(sv, tk, wait=True, nrhs=len(q[2]), want_solution=False)[0]
               for tk, q in zip(tickets, reqs)]
    finally:
        mm.mm_server_destroy(sv)
    assert all(r["status"] == 0 and r["converged"] for r in out)
    # with room for one at a time, requests ran one after another
    starts = sorted(r["queue_s"] for r in out)
    assert starts[-1] > 0


def test_concurrent_requests_of_different_widths_all_converge(family):
    """Four workers, requests of 1 and 16 right-hand sides interleaved: solvers of
    different sizes run their Arnoldi steps concurrently on separate streams and
    all converge (a per-kernel launch attribute shared by them must not be
    lowered by one solver under another's launch)."""
    g = wl.rng(4, 2)
    reqs = []
    for i in range(8):
        side = 3 + (i % 2)
        nrhs = 16 if i % 2 == 0 else 1
        lay = wl.loop_array(side, side, outers=OUTERS, config_index=2)
        type_of = g.integers(0, 4, size=side * side)
        th = g.uniform(0, np.pi / 3, nrhs)
        ph = g.uniform(0, np.pi / 2, nrhs)
        pol = g.integers(0, 2, nrhs)
        reqs.append((type_of, lay.offsets, th, ph, pol, 1e-4))
    sv = mm.mm_server_create(0, workers=4)
    try:
        tickets = [_submit(sv, family, r) for r in reqs]
        for t, r in zip(tickets, reqs):
            res, _ = mm.mm_server_poll(sv, t, wait=True, nrhs=len(r[2]), want_solution=False)
            assert res["status"] == mm.MM_OK and res["converged"], res
            assert res["rel_residual"] <= 1e-4
            mm.mm_server_release(sv, t)
    finally:
        mm.mm_server_destroy(sv)
