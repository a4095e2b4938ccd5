// Library special case used to pin the CPU oracle: the same operation script
// run through std::unordered_map / std::unordered_set.  Reads lines
//   kind
//   I key val | F key | E key | S | C
// and prints one result line per operation.  Keys and values are unsigned
// 64-bit bit patterns.  Capacity is not modelled here: scripts given to this
// program never exceed it.
#include <cstdint>
#include <iostream>
#include <string>
#include <unordered_map>
#include <unordered_set>

int main() {
    int kind;
    if (!(std::cin >> kind)) return 1;
    const bool is_map = kind >= 2;
    std::unordered_map<uint64_t, uint64_t> m;
    std::unordered_set<uint64_t> s;
    std::string op;
    while (std::cin >> op) {
        if (op == "I") {
            uint64_t k, v;
            std::cin >> k >> v;
            bool ok = is_map ? m.insert({k, v}).second : s.insert(k).second;
            std::cout << (ok ? 0 : 1) << "\n";
        } else if (op == "F") {
            uint64_t k;
            std::cin >> k;
            if (is_map) {
                auto it = m.find(k);
                if (it == m.end()) std::cout << "0 0\n";
                else std::cout << "1 " << it->second << "\n";
            } else {
                std::cout << (s.count(k) ? "1 0" : "0 0") << "\n";
            }
        } else if (op == "E") {
            uint64_t k;
            std::cin >> k;
            size_t c = is_map ? m.erase(k) : s.erase(k);
            std::cout << (c ? 3 : 4) << "\n";
        } else if (op == "S") {
            std::cout << (is_map ? m.size() : s.size()) << "\n";
        } else if (op == "C") {
            m.clear();
            s.clear();
            std::cout << "ok\n";
        }
    }
    return 0;
}
