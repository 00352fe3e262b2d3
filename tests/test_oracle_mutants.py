"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of the oracle's C source (a dropped
term, a wrong index or sign, an off-by-one in the stopping rule ...), builds
it into a temporary library and runs the pin tests against it in a child
process: every mutant must make at least one pin fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hanf_oracle.c")

MUTANTS = {
    "union_drops_own_counter": ("memcpy(mv, c_t + v * m, (size_t)m);", "memset(mv, 0, (size_t)m);"),
    "union_min_not_max": ("if (cw[i] > mv[i]) mv[i] = cw[i];", "if (cw[i] < mv[i]) mv[i] = cw[i];"),
    "index_low_bits": ("(h >> (64 - b))", "(h & ((1ULL << b) - 1))"),
    "rho_off_by_one": ("if (bit) { r = i + 1; break; }", "if (bit) { r = i; break; }"),
    "no_rho_clamp": ("if (r > 31) r = 31;", ""),
    "no_linear_counting": ("if (E <= 2.5 * (double)m && V > 0)", "if (0)"),
    "alpha64_wrong": ("if (m == 64) return 0.709;", "if (m == 64) return 0.7213;"),
    "sum_skips_node0": ("for (v = 0; v < n; ++v) {\n        double x = ora_size(",
                        "for (v = 1; v < n; ++v) {\n        double x = ora_size("),
    "stop_one_pass_late": ("if (changed == 0) break;", "if (changed == 0) { if (t < cap - 1) { ++t; N_out[t] = N_out[t - 1]; } break; }"),
    "stop_one_pass_early": ("if (changed == 0) break;\n        ++t;", "++t;\n        if (changed <= 1) break;"),
    "variance_sign": ("out[3] = sq - mean * mean;", "out[3] = sq + mean * mean;"),
    "ied_wrong_side": ("(alpha - prevH) / (H - prevH)", "(H - alpha) / (H - prevH)"),
    "hash_constant_typo": ("0xBF58476D1CE4E5B9ULL", "0xBF58476D1CE4E5B8ULL"),
    "hash_seed_added_not_xored": ("ora_splitmix64(v ^ seed)", "ora_splitmix64(v + seed)"),
    "sizes_skip_node0": ("for (v = 0; v < n; ++v)\n        out[v] = ora_size(",
                         "for (v = 1; v < n; ++v)\n        out[v] = ora_size("),
    "neumaier_drops_branch": ("else comp += (x[i] - t) + s;", "else comp += 0.0;"),
    "digest_drops_node_id": ("buf[i] = (uint8_t)((uint64_t)v >> (8 * i));", "buf[i] = 0;"),
    "fnv_prime_typo": ("h *= 1099511628211ULL;", "h *= 1099511628213ULL;"),
    "seq_radius_strict": ("if (r < 0 && E[t] >= alpha * last) r = t;",
                          "if (r < 0 && E[t] > alpha * last) r = t;"),
    "seq_ecc_previous_pass": ("            e = t;\n", "            e = t - 1;\n"),
    "seq_dist_weight_off_by_one": ("s = s + (double)t * (E[t] - E[t - 1]);",
                                   "s = s + (double)(t - 1) * (E[t] - E[t - 1]);"),
    "ball_radius_off_by_one": ("if (r >= 0 && dist[u] >= r) continue;", "if (r >= 0 && dist[u] > r) continue;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique for {name}"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                    "-shared", "-fvisibility=hidden", "-o", str(lib), str(mut), "-lm"],
                   check=True)
    env = dict(os.environ, HANF_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-k", "not theorem1 and not placement_laws and not estimates_cardinality"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
