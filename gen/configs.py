"""Workload geometry: field sizes, member counts, seeds and region boxes.

Boxes are half-open (x0, y0, z0, x1, y1, z1) in voxels. These are input
recipes only (sizes of the paper's workloads, Section 5.1 and 5.4), no method
arithmetic.
"""

# Small plain-method case: 16x16x4 grid, 32 members, all 523,776 unique pairs,
# 8 regions of 8x8x2 -> 36 region pairs including self.
SMALL = dict(name="small-16x16x4-n32", seed=1, X=16, Y=16, Z=4, n=32, k=3, bins=8,
             region=(8, 8, 2))

# Focus refinement at paper-like scale: two 32x32x20 regions (20,480 points
# each) cut from a 352x256x20 field with 100 members; all 419,430,400 cross
# pairs for Pearson/Spearman, 2,000,000 sampled pairs for KSG (k=10) and
# 16x16-bin histogram MI.
FOCUS = dict(name="focus-352x256x20-n100", seed=2, X=352, Y=256, Z=20, n=100, k=10, bins=16,
             box_a=(64, 64, 0, 96, 96, 20), box_b=(256, 160, 0, 288, 192, 20),
             sampled_pairs=2_000_000, sampler_seed=7)

# Precision case: the same two regions with 1000 members (only the two boxes
# are generated), KSG k=10 on 1,000,000 sampled pairs, top 4096 re-evaluated.
PRECISION = dict(name="precision-2x32x32x20-n1000", seed=2, X=352, Y=256, Z=20, n=1000, k=10,
                 box_a=(64, 64, 0, 96, 96, 20), box_b=(256, 160, 0, 288, 192, 20),
                 sampled_pairs=1_000_000, sampler_seed=7, topk=4096)

# Batched context view: 340x250x20, 100 members, 32x32x20 regions with smaller
# boundary regions (11 x 8 = 88 regions, 3916 region pairs incl. self),
# 30 BOS rounds of 32 candidates per region pair.
CONTEXT = dict(name="context-340x250x20-n100", seed=3, X=340, Y=250, Z=20, n=100, k=10,
               bins=16, region=(32, 32, 20), rounds=30, per_round=32)

# Inter-variable matrix on the context grid: the second variable is 0.6 x the
# first moved by (40, 0) voxels plus 0.8 x an independent seed-5 field; BOS
# over all 88 x 88 ordered region pairs (7744 entries, none symmetric).
INTER_VARIABLE = dict(name="intervar-340x250x20-n100", second_seed=5, shift=(40, 0),
                      rounds=30, per_round=32, check_entries=64)

# Learned surrogate: trained on a seed-2 352x256x20 n=100 field, evaluated on a
# seed-4 field with the focus geometry.
SURROGATE = dict(name="surrogate-352x256x20-n100", train_seed=2, eval_seed=4, X=352, Y=256,
                 Z=20, n=100, k=10, train_pairs=4_000_000, screen_topk=8192,
                 box_a=(64, 64, 0, 96, 96, 20), box_b=(256, 160, 0, 288, 192, 20))


def regular_boxes(X, Y, Z, bx, by, bz):
    """Axis-aligned partition into bx x by x bz boxes; boundary boxes are smaller.

    Enumeration order: x fastest, then y, then z.
    """
    out = []
    for z0 in range(0, Z, bz):
        for y0 in range(0, Y, by):
            for x0 in range(0, X, bx):
                out.append((x0, y0, z0, min(x0 + bx, X), min(y0 + by, Y), min(z0 + bz, Z)))
    return out
