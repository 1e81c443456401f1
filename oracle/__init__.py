"""FP64 CPU oracle for ball-harmonic rotational matching.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, tables or constants with the CUDA library; the only module both sides
use is the seeded input generator ``paper_2509_01180_gb300.synth``, which holds
none of the method's arithmetic.

Modules
-------
``ball``    the basis psi_klm = c_lk j_l(lambda_lk r) Y_l^m chi_[0,1)(r)
            (Sec. II-A, unnumbered display) and the voxel expansion of a volume
            into f_hat_klm (Sec. II-A expansion display).
``wigner``  angular-momentum generators and the Wigner matrices D^l(g)
            (Sec. II-A steerability; Eq. 2).
``align``   xi^l_{mm'}, the rotational cross-correlation of Eq. 2 restricted
            to s = 0, its closed-form derivative (Sec. II-C), multi-start
            gradient ascent with frequency marching (Sec. II-C), the energy
            ratio of Fig. 1, and the final selection.

Everything is FP64 (complex128).  Where the paper is silent the oracle takes
the readings listed at the top of each module; every function names the
passage it follows.
"""
