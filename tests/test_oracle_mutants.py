"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (on the CPU;
the copy is compiled into a temporary library), swaps it in, and runs the pins
of tests/test_oracle_pins.py: at least one must fail.  This is what makes the
pins evidence that the oracle computes the paper's step and not something
close to it.
"""
import pytest

import oracle
import test_oracle_adjoint as adj_pins
import test_oracle_pins as pins

# (name, text in titan_oracle.c, replacement)
MUTANTS = [
    ("force sign on i", "F[3 * i + a] += f * u[a];", "F[3 * i + a] -= f * u[a];"),
    ("reaction on the wrong mass", "F[3 * j + a] -= f * u[a];", "F[3 * i + a] -= f * u[a];"),
    ("rest length dropped", "sys->k[s] * (len - L)", "sys->k[s] * (len)"),
    ("damping dropped", "sys->k[s] * (len - L) + sys->damping[s] * rate",
     "sys->k[s] * (len - L)"),
    ("damping along the velocity difference",
     "F[3 * i + a] += f * u[a];\n            F[3 * j + a] -= f * u[a];",
     "F[3 * i + a] += sys->k[s] * (len - L) * u[a] + sys->damping[s] * dv[a];\n"
     "            F[3 * j + a] -= sys->k[s] * (len - L) * u[a] + sys->damping[s] * dv[a];"),
    ("transposed component", "d[a] = x[3 * j + a] - x[3 * i + a];",
     "d[a] = x[3 * j + (a + 1) % 3] - x[3 * i + (a + 1) % 3];"),
    ("position-first integration",
     "vi[c] = vi[c] + a[c] * dt;\n            xi[c] = xi[c] + vi[c] * dt;",
     "xi[c] = xi[c] + vi[c] * dt;\n            vi[c] = vi[c] + a[c] * dt;"),
    ("forward Euler", "vi[c] = vi[c] + a[c] * dt;\n            xi[c] = xi[c] + vi[c] * dt;",
     "double vo = vi[c];\n            vi[c] = vi[c] + a[c] * dt;\n            xi[c] = xi[c] + vo * dt;"),
    ("gravity sign", "/ m + sys->gravity[c];", "/ m - sys->gravity[c];"),
    ("contact sign", "a[2] += Fn / m;", "a[2] -= Fn / m;"),
    ("friction sign", "a[0] -= fr / m * (vi[0] / vt);", "a[0] += fr / m * (vi[0] / vt);"),
    ("friction cap dropped", "if (cap < fr) fr = cap;", ""),
    ("fixed masses ignored", "if (sys->fixed && sys->fixed[i])", "if (0)"),
    ("actuation phase sign", "* t + sys->act_b[s]", "* t - sys->act_b[s]"),
    ("actuation 2 pi dropped", "2.0 * kPi * sys->act_freq * t", "sys->act_freq * t"),
    ("actuation time off by one step", "(double)step * sys->dt", "(double)(step + 1) * sys->dt"),
    ("adjoint: dashpot sign", "vb[3 * j + a] += rateb * u[a];", "vb[3 * j + a] -= rateb * u[a];"),
    ("adjoint: friction branch", "if (!capped) xbi[2] +=", "if (capped) xbi[2] +="),
    ("adjoint: phase derivative", "sys->act_a[s] * cos(th);", "sys->act_a[s] * sin(th);"),
    ("adjoint: velocity passes dt", "vtot[c] = vb_out[3 * i + c] + dt * xb_out[3 * i + c];",
     "vtot[c] = vb_out[3 * i + c];"),
    ("worm modulo truncated", "tau = tau - sys->worm_period * floor(tau / sys->worm_period);",
     "tau = fmod(tau, sys->worm_period);"),
]

PINS = [getattr(pins, n) for n in dir(pins) if n.startswith("test_")]
PINS += [getattr(adj_pins, n) for n in dir(adj_pins) if n.startswith("test_")]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, tmp_path):
    src = oracle.source()
    # the forward step comes first in the file; a text that the adjoint repeats
    # is mutated at its first (forward) occurrence only
    assert src.count(old) >= 1, f"mutation site for '{name}' not found"
    caught = []
    with oracle.mutant(src.replace(old, new, 1), str(tmp_path)):
        for fn in PINS:
            try:
                if "ground" in fn.__code__.co_varnames[:fn.__code__.co_argcount]:
                    fn(True)
                    fn(False)
                else:
                    fn()
            except (AssertionError, FloatingPointError, ValueError):
                caught.append(fn.__name__)
                break
    assert caught, f"no pin caught mutant '{name}'"
