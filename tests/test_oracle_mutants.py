"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of ``oracle/oracle.c`` (on the CPU),
builds it into a separate library, and runs the pin suite against it in a
subprocess; the suite has to fail.  This checks the pins, not the CUDA path.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "dice_drops_factor_two": ("(double)(2u * inter) / (double)denom", "(double)(inter) / (double)denom"),
    "threshold_strict": ("static int in_mask_f32(float c, float t) { return c >= t; }",
                         "static int in_mask_f32(float c, float t) { return c > t; }"),
    "empty_pair_is_zero": ("if (denom == 0) return 1.0;", "if (denom == 0) return 0.0;"),
    "tie_prefers_high_index": ("if (a->index < b->index) return -1;\n    if (a->index > b->index) return 1;",
                               "if (a->index < b->index) return 1;\n    if (a->index > b->index) return -1;"),
    "flair_uses_t1gd_patient_mask": ("            i2 += m2 & pmask[v + x];\n        }\n        out[4 * e + 0] = i1;\n        out[4 * e + 1] = i2;\n        out[4 * e + 2] = e1;\n        out[4 * e + 3] = e2;\n    }\n    (void)nthreads;\n    return 0;\n}\n\nint oracle_counts_f16",
                                     "            i2 += m2 & pmask[x];\n        }\n        out[4 * e + 0] = i1;\n        out[4 * e + 1] = i2;\n        out[4 * e + 2] = e1;\n        out[4 * e + 3] = e2;\n    }\n    (void)nthreads;\n    return 0;\n}\n\nint oracle_counts_f16"),
    "score_doubles_one_term": ("return (d1 + d2) * 0.5;", "return (d1 + d1) * 0.5;"),
    "f16_exponent_off_by_one": ("expo - 25", "expo - 24"),
    "block_mean_transposed": ("out[bx + bx_n * (by + by_n * bz)]", "out[by + by_n * (bx + bx_n * bz)]"),
    "unpack_bit_reversed": (">> (x % 32)) & 1u", ">> (31 - x % 32)) & 1u"),
    "bf16_rounds_half_up": ("b += 0x7FFFu + lsb;", "b += 0x8000u;"),
    "e4m3_scale_wrong_max": ("float s = (m == 0.0f) ? 1.0f : m / 448.0f;",
                             "float s = (m == 0.0f) ? 1.0f : m / 240.0f;"),
    "e4m3_subnormal_exponent": ("mag = ldexp((double)frac, -9);", "mag = ldexp((double)frac, -10);"),
    "sketch_bucket_bits": ("const int bucket = (int)((h >> 32) & (uint64_t)(d - 1));",
                           "const int bucket = (int)((h >> 33) & (uint64_t)(d - 1));"),
    "sketch_sign_flipped": ("out[bucket] += ((h >> 31) & 1u) ? -1 : 1;",
                            "out[bucket] += ((h >> 31) & 1u) ? 1 : -1;"),
    "sign_code_ge_zero": ("if (sk[j] > 0) code[j / 32]", "if (sk[j] >= 0) code[j / 32]"),
    "rd_face_arithmetic_mean": ("return (a + b > 0.0) ? 2.0 * a * b / (a + b) : 0.0;",
                                "return 0.5 * (a + b);"),
    "rd_reaction_sign": ("rho * ui * (1.0 - ui)", "rho * ui * (1.0 + ui)"),
    "rd_drops_plus_z_flux": ("                    if (z < nz - 1) flux += rd_face(mi, tissue[i + sz]) * (u[i + sz] - ui);\n", ""),
    "rd_dt_off_by_one": ("t_end / (double)n : 0.0;", "t_end / (double)(n + 1) : 0.0;"),
    "rd_y_stride_is_ny": ("const int64_t sy = nx, sz = (int64_t)nx * ny;",
                          "const int64_t sy = ny, sz = (int64_t)nx * ny;"),
    "rd_steps_ignore_m_max": ("double rate = 6.0 * dw * m_max + rho;", "double rate = 6.0 * dw + rho;"),
    "counts_masks_flair_vs_t1gd_patient": ("            i2 += m[v + x] & pmask[v + x];",
                                           "            i2 += m[v + x] & pmask[x];"),
    "counts_masks_drops_plane_offset": ("            e2 += m[v + x];", "            e2 += m[x];"),
    "patient_flair_at_t1": ("        mask[v + x] = (uint8_t)in_mask_f32(vol[x], t2);",
                            "        mask[v + x] = (uint8_t)in_mask_f32(vol[x], t1);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mutated = tmp_path / "oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", str(mutated), "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, DBQ_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_embed_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_sketch_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_rd_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
