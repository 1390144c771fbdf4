"""The C ABI on the host: the library loads, exports every entry point include/lb.h
declares, and validates its arguments; the host-side chain generator.  None of these calls
touches a GPU."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lb_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol(lblib):
    names = _declared()
    assert {"lb_create", "lb_add_chain", "lb_step", "lb_get_populations", "lb_get_beads"} <= names
    for n in names:
        assert hasattr(lblib._lib, n), n


def test_create_validates_arguments(lblib):
    bad = [dict(L=3), dict(rho=0.0), dict(eta=-1.0), dict(eta_b=0.0), dict(kT=-1.0), dict(h=0.0),
           dict(a=0.0), dict(precision=7), dict(precision=100)]
    base = dict(L=8, rho=1.0, eta=3.0, eta_b=3.0, kT=1.0, h=0.01, a=1.0, seed=1, precision=lblib.LB_FP32)
    for b in bad:
        kw = dict(base, **b)
        with pytest.raises(lblib.LBError) as ei:
            lblib.lb_create(**kw)
        assert ei.value.code == lblib.LB_ERR_ARG, b
    ctx = lblib.lb_create(**base)
    lblib.lb_destroy(ctx)


def test_add_chain_validates_and_generates(lblib):
    ctx = lblib.lb_create(16, 1.0, 3.0, 3.0, 1.0, 0.01, 1.0, 7, lblib.LB_FP32)
    try:
        for kw in (dict(N=0), dict(N=1025), dict(N=4, m=0.0), dict(N=4, R0=-1.0)):
            args = dict(N=4, m=1.0, zeta=20.8, k_fene=30.0, R0=1.5, eps=1.0, sigma=1.0)
            args.update(kw)
            with pytest.raises(lblib.LBError) as ei:
                lblib.lb_add_chain(ctx, **args)
            assert ei.value.code == lblib.LB_ERR_ARG
        with pytest.raises(lblib.LBError) as ei:  # generated walk needs bond < R0
            lblib.lb_add_chain(ctx, 4, 1.0, 20.8, 30.0, 1.5, 1.0, 1.0, bond=1.6)
        assert ei.value.code == lblib.LB_ERR_ARG
        with pytest.raises(lblib.LBError) as ei:  # stretched initial bond
            lblib.lb_add_chain(ctx, 2, 1.0, 20.8, 30.0, 1.5, 1.0, 1.0, x0=[[1, 1, 1], [2.6, 1, 1]])
        assert ei.value.code == lblib.LB_ERR_FENE
        lblib.lb_add_chain(ctx, 64, 1.0, 20.8, 30.0, 1.5, 1.0, 1.0, bond=0.97, saw=1)
        with pytest.raises(lblib.LBError) as ei:
            lblib.lb_add_chain(ctx, 4, 1.0, 20.8, 30.0, 1.5, 1.0, 1.0)
        assert ei.value.code == lblib.LB_ERR_STATE
        x = np.empty((64, 3))
        v = np.empty((64, 3))
        lblib.lb_get_beads(ctx, x, v, x.size)
        bonds = np.linalg.norm(np.diff(x, axis=0), axis=1)
        assert np.allclose(bonds, 0.97, rtol=1e-12)
        d = np.linalg.norm(x[:, None] - x[None], axis=-1)
        nonadj = ~np.eye(64, dtype=bool) & ~np.eye(64, k=1, dtype=bool) & ~np.eye(64, k=-1, dtype=bool)
        assert d[nonadj].min() >= 1.0 - 1e-12
        assert np.allclose(x[0], 8.0) and np.all(v == 0)
    finally:
        lblib.lb_destroy(ctx)


def test_workspace_size_accounts_for_precision_and_size(lblib):
    sizes = {}
    for prec in (lblib.LB_FP64, lblib.LB_FP32, lblib.LB_BF16):
        ctx = lblib.lb_create(32, 1.0, 3.0, 3.0, 1.0, 0.01, 1.0, 1, prec)
        sizes[prec] = lblib.lb_workspace_size(ctx)
        lblib.lb_destroy(ctx)
    pop = lambda b: 2 * 19 * 32 ** 3 * b
    assert sizes[lblib.LB_FP64] >= pop(8) and sizes[lblib.LB_FP64] < pop(8) * 1.1
    assert sizes[lblib.LB_FP32] >= pop(4) and sizes[lblib.LB_FP32] < pop(4) * 1.1
    assert sizes[lblib.LB_BF16] >= pop(2) and sizes[lblib.LB_BF16] < pop(2) * 1.2


def test_strerror_names_every_status(lblib):
    for code in range(8):
        assert lblib.lb_strerror(code) != "unknown status"
    assert lblib.lb_strerror(99) == "unknown status"


def test_analysis_and_recording_validate_arguments(lblib):
    """Argument checks run before any launch (no GPU needed)."""
    for call in (lambda: lblib.lb_analysis_msd(None, 10, 4, 3, 1, 2, None, None),
                 lambda: lblib.lb_analysis_msd(1, 10, 4, 3, 1, 4, 1, None),  # i1 out of range
                 lambda: lblib.lb_analysis_rouse_modes(1, 10, 1, 1, 1, None),  # N < 2
                 lambda: lblib.lb_analysis_rouse_modes(1, 10, 4, 4, 1, None),  # P > N-1
                 lambda: lblib.lb_analysis_rouse_correlation(1, 10, 3, 70000, 1, None),
                 lambda: lblib.lb_analysis_static_sk(1, 10, 4, None, 2, 1, None),
                 lambda: lblib.lb_analysis_dynamic_sk(1, 10, 4, 1, 2, 3, 0, 1, None)):  # stride 0
        with pytest.raises(lblib.LBError) as ei:
            call()
        assert ei.value.code == lblib.LB_ERR_ARG
    ctx = lblib.lb_create(8, 1.0, 3.0, 3.0, 1.0, 0.01, 1.0, 1, lblib.LB_FP32)
    with pytest.raises(lblib.LBError) as ei:  # no chain to record
        lblib.lb_record_trajectory(ctx, 1, 4, 1)
    assert ei.value.code == lblib.LB_ERR_STATE
    assert lblib.lb_trajectory_frames(ctx) == 0
    lblib.lb_destroy(ctx)


def test_chain_contexts_add_two_dense_correction_fields(lblib):
    """With a chain, the deferred force corrections live in two dense fields of the
    arithmetic type (FP32 for the 16-bit storage) beside the two population buffers."""
    from paper_0903_5067_gb300 import inputs

    L = 32
    pop = lambda b: 19 * L ** 3 * b
    for prec, s_b, r_b in ((lblib.LB_FP64, 8, 8), (lblib.LB_FP32, 4, 4), (lblib.LB_BF16, 2, 4)):
        ctx = lblib.lb_create(L, 1.0, 3.0, 3.0, 1.0, 0.01, 1.0, 1, prec)
        lblib.lb_add_chain(ctx, 16, 1.0, 20.8, 30.0, 1.5, 1.0, 1.0,
                           x0=inputs.chain_walk(16, L=L, seed=1, self_avoiding=True))
        size = lblib.lb_workspace_size(ctx)
        lblib.lb_destroy(ctx)
        expect = 2 * pop(s_b) + 2 * pop(r_b)
        assert expect <= size < expect * 1.1, prec


def test_inverse_radius_validates_arguments(lblib):
    for call in (lambda: lblib.lb_analysis_inverse_radius(None, 10, 4, 1, None),
                 lambda: lblib.lb_analysis_inverse_radius(1, 10, 1, 1, None)):  # N < 2
        with pytest.raises(lblib.LBError) as ei:
            call()
        assert ei.value.code == lblib.LB_ERR_ARG


def test_bd_create_validates_arguments(lblib):
    x = np.zeros((1, 4, 3))
    base = dict(replicas=1, N=4, kT=1.2, zeta=15.5, eta_s=2.4, dt=0.003, k_fene=7.0, R0=2.0, eps=1.0, sigma=1.0,
                hi=1, degree=20, power_iters=20, seed=1, x0=x, precision=lblib.LB_FP32)
    for bad in (dict(degree=0), dict(degree=65), dict(power_iters=0), dict(kT=0.0), dict(precision=2),
                dict(N=80, x0=np.zeros((1, 80, 3))), dict(N=53, x0=np.zeros((1, 53, 3)), precision=lblib.LB_FP64)):
        with pytest.raises(lblib.LBError) as ei:
            lblib.lb_bd_create(**dict(base, **bad))
        assert ei.value.code == lblib.LB_ERR_ARG, bad


def test_batch_options_before_first_use(lblib):
    """lb_batch_set_options is taken before the batch's first use (no GPU needed) and checks
    its handle."""
    b = lblib.lb_batch_create([8, 12], [0, 0], [1, 2], 1.0, 3.0, 3.0, 1.0, 0.01, 1.0, 1.0, 20.8, 30.0, 1.5, 1.0,
                              1.0, None, lblib.LB_FP32, 1)
    try:
        lblib.lb_batch_set_options(b, 1, 1, 1)
        lblib.lb_batch_set_options(b, 0, 1, 0)
    finally:
        lblib.lb_batch_destroy(b)
    assert lblib._lib.lb_batch_set_options(None, 1, 1, 1) == lblib.LB_ERR_ARG


def test_binding_refuses_buffers_the_library_would_overrun(lblib):
    """The C calls write as many doubles as the capacity they are given; the binding checks
    every caller-owned array against that before the call (dtype, layout, size)."""
    ctx = lblib.lb_create(8, 1.0, 3.0, 3.0, 1.0, 0.01, 1.0, 3, lblib.LB_FP32)
    try:
        with pytest.raises(ValueError):
            lblib.lb_add_chain(ctx, 4, 1.0, 20.8, 30.0, 1.5, 1.0, 1.0, x0=np.zeros((3, 3)))
        with pytest.raises(ValueError):
            lblib.lb_set_options(ctx, ext_bead_force=[1.0, 2.0])
        lblib.lb_add_chain(ctx, 4, 1.0, 20.8, 30.0, 1.5, 1.0, 1.0)
        good = np.empty((4, 3))
        for bad in (np.empty((4, 3), dtype=np.float32), np.empty((3, 4)).T, np.empty((3, 3))):
            with pytest.raises(ValueError):
                lblib.lb_get_beads(ctx, bad, good, 12)
            with pytest.raises(ValueError):
                lblib.lb_get_beads(ctx, good, bad, 12)
        ro = np.empty((4, 3))
        ro.flags.writeable = False
        with pytest.raises(ValueError):
            lblib.lb_get_beads(ctx, ro, None, 12)
        with pytest.raises(ValueError):
            lblib.lb_get_populations(ctx, np.empty((19, 8, 8, 8), dtype=np.float32))
        lblib.lb_get_beads(ctx, good, None, 12)  # the well-formed call still goes through
    finally:
        lblib.lb_destroy(ctx)
    with pytest.raises(ValueError):
        lblib.lb_batch_create([8], [4], [1], 1.0, 3.0, 3.0, 1.0, 0.01, 1.0, 1.0, 20.8, 30.0, 1.5, 1.0, 1.0,
                              np.zeros(9), lblib.LB_FP32)
    with pytest.raises(ValueError):
        lblib.lb_batch_get_populations(None, 0, np.empty(10, dtype=np.float32))
    with pytest.raises(ValueError):
        lblib.lb_bd_get_beads(None, np.empty(10, dtype=np.float32))


def test_failing_calls_leave_a_message_for_their_thread(lblib):
    """lb_last_error hands over the reason of the calling thread's last failure once; the
    binding's LBError carries it."""
    import threading

    assert lblib.lb_last_error() == ""
    with pytest.raises(lblib.LBError) as ei:
        lblib.lb_create(3, 1.0, 3.0, 3.0, 1.0, 0.01, 1.0, 1, lblib.LB_FP32)
    assert "L out of range" in ei.value.detail and "L out of range" in str(ei.value)
    assert lblib.lb_last_error() == ""  # taken by the exception
    import ctypes

    out = ctypes.c_void_p()
    assert lblib._lib.lb_create(ctypes.byref(out), 8, -1.0, 3.0, 3.0, 1.0, 0.01, 1.0, 1, lblib.LB_FP32) != lblib.LB_OK
    seen = []
    t = threading.Thread(target=lambda: seen.append(lblib.lb_last_error()))
    t.start()
    t.join()
    assert seen == [""]  # another thread's failure is not visible here
    msg = lblib.lb_last_error()
    assert "must be > 0" in msg
    n = lblib._lib.lb_last_error(None, 0)
    assert n == 0
    with pytest.raises(lblib.LBError) as ei:  # a null handle
        lblib.lb_step(None, 1)
    assert "invalid argument" in ei.value.detail
