"""Host-side parts of the channel case (no GPU): Eq. error as the product
computes it against the oracle's definition, and the atom count of the
full-channel MD that Eq. speedup divides by, against a hand count."""
import math

import numpy as np

from oracle import hybrid as ohy


def test_channel_error_matches_the_oracle_definition():
    from paper_1603_04628_gb300 import cases
    rng = np.random.default_rng(3)
    Q = rng.normal(2.0, 1.0, 100)
    q = Q + rng.normal(0.0, 0.1, 100)
    assert cases.error(q, Q) == ohy.relative_error(q, Q)
    assert cases.error(Q, Q) == 0.0


def test_full_channel_atom_count_by_hand():
    # 3 sections of dx = 10 under h0 = 12: h = 12 (1 - cos(2 pi j / 3) / 2)
    # = 6, 15, 15; fluid n0 Lz dx sum(h) = 0.8 * 10 * 10 * 36 = 2880.  Two
    # walls of three FCC (100) planes at wall density 1 (lattice constant
    # 4^(1/3), two atoms per plane cell) over 30 x 10: 2 * 3 * 2 * 300 / 4^(2/3)
    from paper_1603_04628_gb300 import cases
    p = dict(n_sections=3, dx=10.0, h0=12.0, Lz=10.0, eos_n0=0.8)
    expect = 2880.0 + 3600.0 / 4.0 ** (2.0 / 3.0)
    assert math.isclose(cases.channel_atoms(p), expect, rel_tol=1e-12)
