"""CPU oracle of the hybrid scheme's hot path: plain, slow, FP64 code written
from the paper (micro-element MD in C, GP, Algorithm 1 and the learned prior
mean in numpy).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
CPU-baseline and reference legs of bench.py may import this package.  It
shares no code with the CUDA library in paper_1603_04628_gb300/."""
