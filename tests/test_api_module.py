"""The module-level calls (fbp, backproject, radon_adjoint, brute_backproject,
fbp_ragged) marshal their arguments into the cached plan's methods.  No GPU:
the plan and batch classes are replaced by recorders whose calls are bound
against the real methods' signatures, so a misnamed or misplaced argument
fails here."""
import inspect

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_1704_08364_gb300 import api  # noqa: E402

RealPlan, RealBatch = api.Plan, api.RaggedBatch


class FakePlan:
    def __init__(self, rays, angles, pad_factor=2):
        inspect.signature(RealPlan.__init__).bind(self, rays, angles, pad_factor)
        self.rays, self.angles, self.pad_factor = int(rays), np.asarray(angles), int(pad_factor)
        self.calls = []

    def __getattr__(self, name):
        sig = inspect.signature(getattr(RealPlan, name))

        def record(*args, **kw):
            sig.bind(self, *args, **kw)
            self.calls.append((name, args, kw))
            return name
        return record


class FakeBatch:
    status_code = 0
    made = []

    def __init__(self, plans):
        self.plans = list(plans)
        self.log = []
        FakeBatch.made.append(self)

    def bind(self, sinos, volumes, gs=None, flags=0):
        inspect.signature(RealBatch.bind).bind(self, sinos, volumes, gs)
        self.log.append(("bind", sinos, volumes, gs))
        return self

    def run(self, use_graph=False):
        self.log.append(("run", use_graph))

    def status(self):
        self.log.append(("status",))
        return FakeBatch.status_code


@pytest.fixture
def fakes(monkeypatch):
    monkeypatch.setattr(api, "Plan", FakePlan)
    monkeypatch.setattr(api, "RaggedBatch", FakeBatch)
    dev = {"i": 0}
    monkeypatch.setattr(api, "_device_index", lambda: dev["i"])
    api.clear_plans()
    FakeBatch.made.clear()
    FakeBatch.status_code = 0
    yield dev
    api.clear_plans()


def test_plans_are_cached_per_device_geometry_and_pad(fakes):
    th = np.arange(8) * np.pi / 8
    p = api.plan_for(16, th, 2)
    assert api.plan_for(16, th.astype(np.float32), 2) is p
    assert api.plan_for(16, th, 1) is not p
    assert api.plan_for(16, th[:7], 2) is not p
    fakes["i"] = 1
    assert api.plan_for(16, th, 2) is not p


def test_calls_reach_the_plan_methods(fakes):
    th = np.arange(8) * np.pi / 8
    sino = torch.zeros(2, 8, 16)
    vol = torch.zeros(2, 16, 16)
    g = torch.ones(16)
    assert api.fbp(sino, th, g=g) == "fbp"
    assert api.backproject(sino, th) == "backproject"
    assert api.radon_adjoint(vol, th, mode=api.BACKPROJECT) == "radon_adjoint"
    assert api.brute_backproject(sino, th, g=g) == "brute_backproject"
    plan = api.plan_for(16, th, 2)
    names = [c[0] for c in plan.calls]
    assert names == ["fbp", "backproject", "radon_adjoint", "brute_backproject"]
    assert plan.calls[0][1][0] is sino and plan.calls[0][2]["g"] is g
    assert plan.calls[2][1][0] is vol and plan.calls[2][2]["mode"] == api.BACKPROJECT
    assert api.fbp(sino[0], th, pad_factor=1) == "fbp" and api.plan_for(16, th, 1).rays == 16


def test_fbp_ragged_pairs_items_of_one_geometry_and_returns_volumes(fakes):
    sinos = [torch.zeros(8, 16), torch.zeros(12, 24), torch.zeros(8, 16)]
    vols = api.fbp_ragged(sinos)
    assert [tuple(v.shape) for v in vols] == [(16, 16), (24, 24), (16, 16)]
    (b,) = FakeBatch.made
    assert b.plans[0] is b.plans[2] and b.plans[0] is not b.plans[1]
    np.testing.assert_allclose(b.plans[1].angles, np.arange(12) * np.pi / 12, rtol=1e-6)
    assert [e[0] for e in b.log] == ["bind", "run", "status"]
    assert b.log[0][2] == vols


def test_fbp_ragged_raises_on_a_device_status(fakes):
    FakeBatch.status_code = 5   # BST_ERR_TIMEOUT
    with pytest.raises(api.BstError):
        api.fbp_ragged([torch.zeros(8, 16)])
