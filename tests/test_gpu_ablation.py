"""Ablation and analytic benchmark on the GPU (Table III, Sec. V-C; Table I
tests; the friction x force sweep of Sec. V-A): removing either modification
of PBD-R must degrade the quantity it protects by a large factor, and PBD-R
must beat standard PBD on every test and sweep point.  Thresholds sit well
below the measured ratios (Test 1: velocity 88x, linear momentum 17x;
Test 2: rotation 94x, angular momentum 3300x)."""
import numpy as np
import pytest

from paper_2603_14634_gb300 import ablation

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def table(pbdr_lib):
    with pbdr_lib.Context(0) as c:
        return ablation.table3(c, T=10.0)


def test_pbdr_tracks_the_closed_forms(table):
    t1, t2 = table["test1"]["PBD-R"], table["test2"]["PBD-R"]
    assert t1["pos"]["end"] < 0.05          # of a 16.3 m slide after 10 s
    assert t1["vel"]["end"] < 0.01          # of 3.26 m/s
    assert t2["rot"]["end"] < 0.1           # degrees, of 286 deg turned after 10 s


def test_velocity_update_ablation(table):
    ab = table["test1"]["no velocity update"]
    assert ab["vel"]["x"] > 10 and ab["pos"]["x"] > 5


def test_linear_momentum_ablation(table):
    ab = table["test1"]["no linear momentum"]
    assert ab["lin"]["x"] > 5 and ab["pos"]["x"] > 3


def test_angular_momentum_ablation(table):
    ab = table["test2"]["no angular momentum"]
    assert ab["rot"]["x"] > 10 and ab["ang"]["x"] > 100


def test_standard_pbd_is_worse(table):
    assert table["test1"]["PBD"]["vel"]["x"] > 10
    assert table["test2"]["PBD"]["rot"]["x"] > 10


def test_tests_1_to_3_pbdr_beats_pbd(pbdr_lib):
    with pbdr_lib.Context(0) as c:
        res = ablation.tests123(c, T=10.0)
    assert res["test1 PBD-R"]["pos"]["end"] < 0.2 * res["test1 PBD"]["pos"]["end"]
    assert res["test2 PBD-R"]["rot"]["end"] < 0.2 * res["test2 PBD"]["rot"]["end"]
    assert res["test3 PBD-R"]["pos"]["end"] < 0.2 * res["test3 PBD"]["pos"]["end"]


def test_friction_force_sweep(pbdr_lib):
    with pbdr_lib.Context(0) as c:
        rows = ablation.sweep(c, mus=(0.1, 0.4), forces=(20.0, 30.0), T=5.0)
    assert len(rows) == 4
    for r in rows:
        assert r["PBD-R pos"] < 0.2 * r["PBD pos"], r
