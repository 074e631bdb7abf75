"""Linear probing with wrap-around over given home slots (Eq. 3's insertion rule), for the
probe-count tests: the model the GPU counts are compared with, and whose order-independence
the CPU tests check."""
import numpy as np


def linear_probing_model(homes, n_slots):
    """Occupied slots and total displacement of linear probing over the given home slots,
    inserted in list order (both are the same for every order), and the longest displacement
    (which is not)."""
    occ = np.zeros(n_slots, bool)
    total = 0
    longest = 0
    for h in homes:
        i, d = h, 0
        while occ[i]:
            i = (i + 1) % n_slots
            d += 1
        occ[i] = True
        total += d + 1
        longest = max(longest, d)
    return occ, total, longest


def miss_reads(occ, home, bound):
    """Slots a lookup of an absent key reads: the run of occupied slots from its home, then the
    empty one, cut at the probe bound."""
    n = occ.size
    run = 0
    while run < n and occ[(home + run) % n]:
        run += 1
    return min(run + 1, bound)
