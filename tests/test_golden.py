"""The golden fixtures under tests/golden/ parse and hold what their citations
say (CPU)."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_table1_fixture():
    """Table 1 (Sec. 3.2): cases 3-18 of the decomposed beam, each with a weight
    type, an overlap width of 1, 3 or 5 dx, Newmark betas in [0, 1/4], m in
    {1, 2, 5, 10} and an error between 0.7 % and 1.8 %; the explicit-PD MTS
    cases (13, 17, 18) are cubic over 3 dx."""
    rows = []
    with open(os.path.join(GOLDEN, "table1_beam_ux_error.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                case, kind, cells, beta_fe, beta_pd, m, err = line.split()
                rows.append((int(case), kind, int(cells), float(beta_fe), float(beta_pd), int(m), float(err)))
    assert [r[0] for r in rows] == list(range(3, 19))
    assert {r[1] for r in rows} == {"constant", "linear", "cubic"}
    assert all(r[2] in (1, 3, 5) and 0 <= r[3] <= 0.25 and 0 <= r[4] <= 0.25 for r in rows)
    assert all(r[5] in (1, 2, 5, 10) and 0.7 <= r[6] <= 1.8 for r in rows)
    explicit_mts = {r[0]: (r[1], r[2], r[5]) for r in rows if r[4] == 0 and r[5] > 1 and r[3] == 0.25}
    assert explicit_mts == {13: ("cubic", 3, 2), 17: ("cubic", 3, 5), 18: ("cubic", 3, 10)}


def test_oracle_plate_run_matches_its_recorded_summary():
    """The oracle's 500-step run of the 100 x 100 pre-cracked plate reproduces
    the summary tests/golden/make_oracle_goldens.py recorded from it (counts
    exactly, the state bit for bit): an unintended change of the oracle's
    arithmetic fails here. The counts are cross-checked by integer arithmetic:
    intact = family - pre-cut - broken."""
    import importlib.util
    import json
    spec = importlib.util.spec_from_file_location("make_oracle_goldens",
                                                  os.path.join(GOLDEN, "make_oracle_goldens.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(os.path.join(GOLDEN, "oracle_plate_100x100.json")) as f:
        rec = json.load(f)
    got = mod.run()
    assert got == rec
    assert rec["intact_at_end"] == rec["directed_bonds"] - rec["precut"] - rec["broken_by_dynamics"]
    assert rec["directed_bonds"] == 272836 and rec["precut"] == 720
