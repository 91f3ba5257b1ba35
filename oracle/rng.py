"""SplitMix64 counter-based generator (oracle copy).  TEST INFRASTRUCTURE ONLY.

The inlet perturbation of the plain cylinder workload is a random number that
both the oracle and the CUDA kernels must draw identically without sharing
code, so each side implements this one published generator on its own.

SplitMix64 is the generator of Steele, Lea and Flood, "Fast splittable
pseudorandom number generators" (OOPSLA 2014): add the golden-ratio increment
0x9E3779B97F4A7C15 to the counter, then apply the 64-bit finaliser
z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
z ^= z >> 31.  Here it is used statelessly: the counter is a key built from the
seed, the time step and the lattice row.
"""

MASK64 = (1 << 64) - 1


def splitmix64(key: int) -> int:
    """One SplitMix64 output for a 64-bit counter value ``key``."""
    z = (key + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def unit_double(z: int) -> float:
    """Top 53 bits of a 64-bit word as a double in [0, 1)."""
    return (z >> 11) * (1.0 / (1 << 53))


def inlet_key(seed: int, t: int, y: int) -> int:
    """Counter for row ``y`` at time step ``t``: seed XOR (t * 2^20 + y)."""
    return (seed ^ ((t << 20) + y)) & MASK64


def inlet_perturbation(seed: int, t: int, ny: int, amp: float):
    """Transverse inlet velocity v(y, t) = amp * (2 xi - 1), xi uniform in [0, 1).

    The paper's cylinder runs shed vortices on their own; the plain cylinder
    workload triggers shedding with a small seeded perturbation of the inlet's
    v, and this is its definition: one draw per inlet row per time step.
    """
    return [amp * (2.0 * unit_double(splitmix64(inlet_key(seed, t, y))) - 1.0)
            for y in range(ny)]
