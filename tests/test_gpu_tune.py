"""The autotuner's search (tile shape, bodies per thread, j-tile and j-split
chosen by timing every compiled variant through the library), run end to end
on small sizes: the table it writes must reload, apply to a context, select
the chosen (variant, split) per size bucket, and the chosen kernels must pass
the same oracle parity as every other force call (float32 compensated:
per-body relative error RMS <= 1e-5, max <= 1e-4; double-float: max <= 1e-12).
"""
import json

import numpy as np
import pytest

import oracle
from paper_1211_2292_gb300 import inputs, nbody, tune
from helpers import host, relerr_per_body, to_dev

pytestmark = pytest.mark.gpu

SIZES = [1024, 4096]


def test_time_candidates_covers_every_variant_and_split(cuda):
    res = tune.time_candidates(nbody.KIND_FORCE, "df64", 1024, splits=(0, 2), reps=1)
    nv = len(nbody.variants(nbody.KIND_FORCE, "df64"))
    assert sorted((v, s) for _, v, s in res) == [(v, s) for v in range(nv) for s in (0, 2)]
    assert all(ms > 0 for ms, _, _ in res)
    assert [ms for ms, _, _ in res] == sorted(ms for ms, _, _ in res)


@pytest.mark.parametrize("prec", ["fp32_comp", "df64"])
def test_autotune_table_applies_and_chosen_kernels_match_oracle(cuda, tmp_path, prec):
    table = tune.autotune(precisions=(prec,), kinds=(nbody.KIND_FORCE,),
                          sizes={nbody.KIND_FORCE: SIZES}, splits=(0, 3), reps=1, batch=False,
                          log=None)
    ent = table["entries"]
    assert [(e["lo"], e["hi"], e["n"]) for e in ent] == [(0, 2048, 1024), (2048, 1 << 40, 4096)]
    path = tmp_path / "table.json"
    path.write_text(json.dumps(table))
    for e in ent:
        assert e["precision"] == prec and e["kind"] == nbody.KIND_FORCE and e["ms"] > 0
        b = inputs.plummer(e["n"], seed=900 + e["n"])
        with nbody.NBody(e["n"], prec) as nb:
            assert tune.apply(nb, str(path)) == len(ent)
            assert nb.tune_get(nbody.KIND_FORCE, e["n"]) == (e["variant"], e["split"])
            a = host(nb.forces(to_dev(b.pos, cuda), to_dev(b.mass, cuda), 1.0, 0.01))
            nb.sync()
        err = relerr_per_body(a, oracle.accel(b.pos, b.mass, 1.0, 0.01))
        if prec == "df64":
            assert err.max() <= 1e-12
        else:
            assert np.sqrt((err ** 2).mean()) <= 1e-5 and err.max() <= 1e-4


def test_packaged_table_covers_every_precision(cuda):
    table = tune.load()
    for prec in ("fp32_comp", "fp32", "fp64", "df64"):
        kinds = {e["kind"] for e in table["entries"] if e["precision"] == prec}
        assert nbody.KIND_FORCE in kinds and nbody.KIND_VJP in kinds, prec
        with nbody.NBody(1024, prec) as nb:
            assert tune.apply(nb, table) > 0
