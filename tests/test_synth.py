"""The seeded input generator (inputs only: no halo-finder arithmetic): reproducible
draws, the recipe's sizes, and the pre-labelled batching workload's labels."""
import numpy as np

import synth


def test_boxes_are_reproducible_and_on_the_lattice():
    a = synth.named("m64")
    b = synth.named("m64")
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.vel, b.vel)
    assert a.pos.min() >= 0 and a.pos.max() < synth.LATTICE
    c = synth.named("m64", replica=1)
    assert not np.array_equal(a.pos, c.pos)
    # 40% of the particles in hosts, the rest uniform background (host_id -1)
    assert abs((a.host_id >= 0).mean() - 0.4) < 0.01


def test_link_length_threshold_is_exact():
    """T = floor(l^2) + 1 with l = 0.2 * 2^21 / m: d^2 < T iff d < l for integer d^2."""
    for m in (32, 64, 256, 512, 1024):
        T = synth.link_d2_for(m ** 3)
        ell = 0.2 * synth.LATTICE / m
        assert (T - 1) < ell * ell < T


def test_prelabelled_halos():
    box, lab = synth.prelabelled_halos(3000, synth.SEED0 + 3, size_hi=1e5)
    sizes = np.bincount(box.host_id)
    assert len(sizes) == 3000 and sizes.min() >= 20 and sizes.max() <= 100000
    assert box.n == sizes.sum() and (box.host_id >= 0).all()  # no background
    # labels: the minimum particle index of each particle's host
    first = np.full(3000, box.n)
    np.minimum.at(first, box.host_id, np.arange(box.n))
    assert np.array_equal(lab, first[box.host_id])
    assert (lab[lab] == lab).all()  # every label is its own halo's member
    # the same seed draws the same halos; the size distribution is the same power law as
    # the mass-function boxes (dN/dM ~ M^-1.9 on [20, size_hi]): about half the hosts
    # below 2^(1/0.9) * 20 ~ 43 members
    box2, lab2 = synth.prelabelled_halos(3000, synth.SEED0 + 3, size_hi=1e5)
    assert np.array_equal(box.pos, box2.pos) and np.array_equal(lab, lab2)
    assert 0.4 < (sizes < 43).mean() < 0.6
