"""Plain, slow FP64 CPU oracle of the kernel-free boundary integral (KFBI)
method for the FitzHugh-Nagumo bidomain equations.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or run this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA library; both read the
seeded inputs of ``kfbi_workloads``.

Modules and the passages they follow:
  levelset  - domains' level sets (bit-exact classification), normals, shape
              operators (Sections 5.3, 6)
  grid      - classification, irregular nodes, crossings, cell indexing
              (Sections 5.3, 6)
  boxsolve  - the 5/7-point system solved by sine transforms (Sections 5.2-5.3)
  density   - psi and its surface gradient: periodic cubic splines (2-D) and
              the six-point local quadratic (3-D) (Sections 5.3, 7)
  kfbi      - jumps, irregular-node correction, Taylor interpolation of the
              limits, the operator A and the right-hand side g (Sections
              4, 5.1-5.4, Algorithm 1)
  krylov    - simple (Richardson) iteration and GMRES (Section 4)
  reaction  - FitzHugh-Nagumo forward/backward Euler half steps (Sections 3, 7)
  bidomain  - the Strang step with the implicit midpoint diffusion and the
              lambda of its decoupled V problem (Section 3, Eq. pde1)
  mlp       - the point-wise network of the learned warm start
  warmstart - history projection, features, prediction and training
              targets of the warm starts (not in the paper)
"""
