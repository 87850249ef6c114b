"""Algorithm 1's pseudoMD (Sec. 2.4): the library's finite-difference
start-up time (mdgp_pseudo_md, host code, no GPU) against the oracle's
eigenfunction series."""
import pytest

from oracle import hybrid as oh


@pytest.fixture(scope="module")
def native():
    from paper_1603_04628_gb300 import build, native as nat
    build.build()
    return nat


CASES = [
    # h, nu, slip, g_from, g_to, from_rest, q_scale, eps_q
    (8.0, 2.5, 0.0, 0.0, 0.02, True, 80.0, 0.05),
    (8.0, 2.5, 0.7, 0.0, 0.02, True, 80.0, 0.05),
    (12.0, 2.2, 0.7, 0.01, 0.02, False, 80.0, 0.05),
    (12.0, 2.2, 0.7, 0.03, 0.02, False, 80.0, 0.01),
    (5.0, 3.0, 2.0, -0.02, 0.04, False, 64.0, 0.1),
    (20.0, 2.0, 0.3, 0.0, 0.005, True, 80.0, 0.02),
    (8.0, 2.5, 50.0, 0.0, 0.02, True, 80.0, 0.5),
    (12.0, 3.1, -0.9, 0.01, 0.03, False, 80.0, 0.05),
]


@pytest.mark.parametrize("case", CASES)
def test_start_up_time_matches_the_series(native, case):
    t_lib = native.pseudo_md(*case)
    t_or = oh.pseudo_md_time(*case)
    h, nu = case[0] + 2 * min(case[2], 0.0), case[1]
    dt = h * h / (nu * 3.141592653589793 ** 2) / 1000.0
    # second order in space (64 cells), first order in time, and t_s lands on the time grid
    assert abs(t_lib - t_or) <= 2e-3 * t_or + 2 * dt, (t_lib, t_or)


def test_no_wait_and_argument_checks(native):
    assert native.pseudo_md(8.0, 2.5, 0.5, 0.02, 0.02, False, 80.0, 0.01) == 0.0
    # the tolerance above the whole jump: nothing to wait for either
    assert native.pseudo_md(8.0, 2.5, 0.5, 0.0, 0.02, True, 80.0, 1e9) == 0.0
    for bad in ((0.0, 2.5, 0.5), (8.0, 0.0, 0.5), (8.0, 2.5, -4.0)):
        with pytest.raises(native.MdgpError):
            native.pseudo_md(*bad, 0.0, 0.02, True, 80.0, 0.01)
