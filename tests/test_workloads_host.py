"""Host-side logic of the benchmark workloads, on the CPU.

The stationary shock (Sec. 5.2) is set up from the Rankine-Hugoniot
relations of a Mach 3 normal shock in a monatomic gas: the end states must
carry equal fluxes of mass, momentum and energy, with the ratios that the
relations give for M = 3 and gamma = 5/3 (density 3, velocity 1/3,
pressure 11, temperature 11/3)."""
import numpy as np
import pytest

from paper_1009_2768_gb300.workloads import rankine_hugoniot


@pytest.mark.parametrize("mach", [1.5, 3.0, 8.0])
def test_rankine_hugoniot_states_carry_equal_fluxes(mach):
    g = 5.0 / 3.0
    (rl, ul, tl), (rr, ur, tr) = rankine_hugoniot(mach)
    pl, pr = rl * tl, rr * tr
    assert abs(ul / np.sqrt(g * tl) - mach) < 1e-12                 # upstream Mach number
    assert abs(rl * ul - rr * ur) < 1e-12 * rl * ul                  # mass
    assert abs((rl * ul * ul + pl) - (rr * ur * ur + pr)) < 1e-12 * (rl * ul * ul + pl)    # momentum
    hl = 0.5 * ul * ul + g / (g - 1.0) * tl                            # specific total enthalpy
    hr = 0.5 * ur * ur + g / (g - 1.0) * tr
    assert abs(rl * ul * hl - rr * ur * hr) < 1e-12 * rl * ul * hl   # energy
    assert ur < ul and pr > pl                                         # a compression shock


def test_mach_3_ratios():
    (rl, ul, tl), (rr, ur, tr) = rankine_hugoniot(3.0)
    assert abs(rr / rl - 3.0) < 1e-12
    assert abs(ur / ul - 1.0 / 3.0) < 1e-12
    assert abs(rr * tr / (rl * tl) - 11.0) < 1e-12
    assert abs(tr / tl - 11.0 / 3.0) < 1e-12


def test_collide_hash_ignores_comments_only(tmp_path, monkeypatch):
    """bench.py keys its ncu records by a hash of the collide sources that
    skips comments and whitespace, and changes with any code."""
    import bench
    d = tmp_path / "paper_1009_2768_gb300" / "csrc"
    d.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))

    def sha(collide):
        (d / "collide.cu").write_text(collide)
        (d / "trmc_device.cuh").write_text("int f(int x) { return x; } // helper\n")
        (d / "fp64_tables.inc").write_text("static const double k = 1.0;\n")
        return bench.collide_sha()

    base = sha("int a = 1; // one\n/* block\n comment */ int b = a + 2;\n")
    assert sha("int a = 1;   // uno\n\nint b = a + 2;  /* another */\n") == base
    assert sha("int a = 1; int b = a + 3;\n") != base
    assert len(base) == 16
