"""Plant plausible mistakes in copies of the oracle and check that the pins catch each.

Every mutant is a textual edit of ``oracle/fw_oracle.c`` compiled into a
temporary library on the CPU; the real oracle is never modified. A mutant
that passed every pin would mean the pins cannot see that kind of mistake.
"""
import os

import pytest

import oracle
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "fw_oracle.c")

MUTANTS = {
    "port_low_exclusive": ("return lo <= port && port <= hi;", "return lo < port && port <= hi;"),
    "port_high_exclusive": ("return lo <= port && port <= hi;", "return lo <= port && port < hi;"),
    "dst_dropped": ("&& address_matches(dst, r->dst_addr, r->dst_prefix)", ""),
    "dport_dropped": ("&& port_matches(dport, r->dport_lo, r->dport_hi)", ""),
    "proto_dropped": ("&& proto_matches(proto, r->proto, r->proto_any)", ""),
    "prefix_off_by_one": ("unsigned drop = 32u - prefix;", "unsigned drop = 33u - prefix;"),
    "proto_any_ignored": ("if (any) return 1;", "if (0) return 1;"),
    "last_match": ("found = (int32_t)k;\n                break;", "found = (int32_t)k;"),
    "default_accept": ("(uint8_t)0 /* DROP: default deny */", "(uint8_t)1"),
    "index_shift": ("found = (int32_t)k;", "found = (int32_t)k + (k > 0);"),
    "ports_swapped": ("port_matches(sport, r->sport_lo, r->sport_hi)", "port_matches(sport, r->dport_lo, r->dport_hi)"),
    "src_uses_dst_prefix": ("address_matches(src, r->src_addr, r->src_prefix)", "address_matches(src, r->src_addr, r->dst_prefix)"),
    "depth_off_by_one": ("(int64_t)found + 1", "(int64_t)found"),
    "unmatched_depth_zero": ("(found < 0) ? n_rules :", "(found < 0) ? 0 :"),
    "address_low_bits": ("uint64_t a = (uint64_t)addr >> drop;\n    uint64_t b = (uint64_t)rule_addr >> drop;",
                         "uint64_t a = ((uint64_t)addr << drop) & 0xFFFFFFFFull;\n"
                         "    uint64_t b = ((uint64_t)rule_addr << drop) & 0xFFFFFFFFull;"),
    "prefix_zero_32bit_shift": ("uint64_t a = (uint64_t)addr >> drop;\n    uint64_t b = (uint64_t)rule_addr >> drop;",
                                "uint64_t a = (uint32_t)(addr >> (drop & 31u));\n"
                                "    uint64_t b = (uint32_t)(rule_addr >> (drop & 31u));"),
    "proto_zero_as_any": ("if (any) return 1;", "if (any || rule_proto == 0) return 1;"),
    "packet_addresses_swapped": ("address_matches(src, r->src_addr", "address_matches(dst, r->src_addr"),
    "packet_ports_swapped": ("port_matches(sport, r->sport_lo", "port_matches(dport, r->sport_lo"),
    "first_rule_skipped": ("for (int64_t k = 0; k < n_rules; ++k)", "for (int64_t k = 1; k < n_rules; ++k)"),
    "last_rule_skipped": ("for (int64_t k = 0; k < n_rules; ++k)", "for (int64_t k = 0; k < n_rules - 1; ++k)"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert old in text, f"mutation site for {name} not found"
    src = tmp_path / f"{name}.c"
    src.write_text(text.replace(old, new, 1))
    lib = oracle.load(oracle.build(str(src), str(tmp_path / f"{name}.so"), force=True))
    failures = []
    for pin in P.ALL_PINS:
        try:
            pin(lib)
        except (AssertionError, IndexError, ValueError):
            failures.append(pin.__name__)
    assert failures, f"mutant {name} passed every pin"
