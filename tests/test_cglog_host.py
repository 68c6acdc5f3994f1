"""Host logic of the per-iteration CGNR log: rates from the per-kind sums."""
import pytest

from paper_2508_10405_gb300.cglog import BYTES_PER_CELL, iteration_record


class FakeOp:
    ndim = 2


def test_iteration_record_rates():
    tm = {"born_ms": 2.0, "born_cells": 4e9, "born_launches": 10,
          "background_ms": 0.0, "background_cells": 0.0, "background_launches": 0,
          "adjoint_ms": 4.0, "adjoint_cells": 4e9, "adjoint_launches": 12}
    r = iteration_record(FakeOp(), 3, 0.5, 1.25, tm, model_error=0.25)
    assert r["iteration"] == 3 and r["misfit"] == 0.5 and r["rel_model_error"] == 0.25
    assert "background" not in r
    # 4e9 cells in 2 ms = 2000 Gcell/s; in 4 ms = 1000 Gcell/s
    assert r["born"]["gcell_per_s"] == pytest.approx(2000.0)
    assert r["adjoint"]["gcell_per_s"] == pytest.approx(1000.0)
    assert r["born"]["gb_per_s"] == pytest.approx(2000.0 * BYTES_PER_CELL[("born", 2)])
    assert r["gcell_per_s"] == pytest.approx(8e9 / 6.0 / 1e6)
    bytes_all = 4e9 * (BYTES_PER_CELL[("born", 2)] + BYTES_PER_CELL[("adjoint", 2)])
    assert r["gb_per_s"] == pytest.approx(bytes_all / 6.0 / 1e6)
