"""Argument handling of the command-line run (no GPU needed): the presets are
the paper's Table A1 runs, and explicit arguments override them."""
import pytest

from paper_2605_25872_gb300.run import PRESETS, parse_args, temperatures


def test_presets_are_the_papers_runs():
    a = parse_args(["--preset", "paper-L16", "--out", "x.jsonl"])
    assert (a.L, a.t_min, a.t_max, a.temps, a.samples, a.emcs) == (16, 0.2, 2.0, 60, 2081, 38_400_000)
    assert a.rule == "metropolis" and a.micsa_bins == 2          # PTHR for bins 2, 3; PTHR* for 0, 1
    a = parse_args(["--preset", "paper-L18", "--out", "x.jsonl"])
    assert a.rule == "micsa" and a.temps == 72 and a.L == 18
    a = parse_args(["--preset", "paper-L12", "--out", "x.jsonl"])
    assert (a.t_min, a.t_max, a.temps, a.emcs) == (0.42, 1.8, 24, 2 ** 17)
    assert set(PRESETS) == {"paper-L12", "paper-L14", "paper-L16", "paper-L18"}


def test_explicit_arguments_override_the_preset_and_defaults_fill_the_rest():
    a = parse_args(["--preset", "paper-L16", "--samples", "64", "--emcs", "1024", "--out", "x.jsonl"])
    assert a.samples == 64 and a.emcs == 1024 and a.temps == 60
    a = parse_args(["--L", "8", "--emcs", "100", "--out", "x.jsonl"])
    assert (a.samples, a.temps, a.t_min, a.t_max, a.rule, a.micsa_bins) == (16, 24, 0.2, 1.6, "metropolis", 0)
    with pytest.raises(SystemExit):
        parse_args(["--out", "x.jsonl"])


def test_temperature_grid_ends_and_spacing():
    T = temperatures(0.2, 2.0, 60)
    assert T[0] == 0.2 and T[-1] == pytest.approx(2.0, abs=1e-15) and len(T) == 60
    assert max(abs((T[1:] - T[:-1]) - 1.8 / 59)) < 1e-14
